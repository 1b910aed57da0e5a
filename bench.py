"""Benchmark of the RK-3 step on the large 2D channel (1024 x 512 nodes,
16 x 8 x 8 = 1024 velocities, FP32, WENO-5, walls T = 1 and 2, Kn = 0.5,
a = (-0.3, -0.3, 0)).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step = one RK-3 step (three wall + three stage kernels) over the whole
grid.  The metric is node-velocity updates per second (a node-velocity update
advances one (node, velocity) value one full RK-3 step).  Prints one JSON
line.  ``--impl reference`` times the FP64 CPU oracle on a bounded sample of
the same workload instead.  Under torchrun each rank runs an independent
replica (the method has no data-parallel split that needs a collective).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1708_03249_gb300 import workloads as W  # noqa: E402

WORKLOAD = "large_2d_channel_1024x512_hhlb8x8x8_weno5_fp32"
METRIC = "node-velocity updates/s"
BYTES_PER_NV_STAGE = 32.0 / 3.0      # FP32: stage 1 reads f^n, writes f1 (8 B); stages 2, 3 read two, write one (12 B)
# FP32 ALU roof: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x the SM clock
SMS, FP32_LANES_PER_SM, MAX_SM_MHZ = 152, 128, 2070.0


FORCE_FORMS = {0: "fma", 1: "tf32x3 tensor cores", 2: "split-bf16 tensor cores"}
PRECISIONS = {"fp32": W.FP32, "tf32x3": W.FP32_TF32X3, "bf16split": W.FP32_BF16SPLIT}


def with_precision(cfg, name: str):
    """The FP32 workload cfg (or list) with the force-term form `name`; FP64 ones unchanged."""
    if isinstance(cfg, list):
        return [with_precision(c, name) for c in cfg]
    if cfg["precision"] == W.FP64:
        return cfg
    return dict(cfg, precision=PRECISIONS[name])


def flops_per_nv_stage(cfg) -> float:
    """Algorithmic flops of one node-velocity in one RK-3 stage: the K_x and
    K_y contractions (2 flop per term), WENO-5 at ~60 flop per spatial axis
    (one face per axis and node-velocity, each shared by two cells), ~20 for
    the moments' share, the equilibrium product, BGK and the RK-3 combination."""
    qx2 = cfg["Qx"] if cfg.get("x_basis", 0) == W.X_FULL else 2 * cfg["Qx"]
    vy = max(cfg["Qy"], 1)
    axes = 2 if cfg["ny"] > 1 else 1
    weno = 60 if cfg["advection"] == W.WENO5 else 4
    if cfg.get("x_basis", 0) == W.X_HALF and cfg["Qx"] > 32:
        # K^h applied as its same-half block plus the rank-one cross-half term
        kx = 2 * cfg["Qx"] + 2
    else:
        kx = 2 * qx2
    return kx + (2 * vy if cfg["Qy"] else 0) + weno * axes + 20


# FP64 roof (no measured figure exists): the nominal 1.25 TFLOP/s of the part
FP64_NOMINAL_TFLOPS = 1.25
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("hlb_pair.cuh", "hlb_pair.cu", "hlb_device.cuh", "hlb_internal.h"):
        with open(os.path.join(ROOT, "paper_1708_03249_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


_FP32_PEAK = None


def fp32_alu_peak(sm_mhz: float):
    """The FP32 ALU roof: the FMA throughput measured on this GPU by the library
    (scalar and packed f32x2 chains, the larger), with the nominal figure (152 SMs
    x 128 FP32 lanes x 2 flop x the SM clock) beside it for context."""
    global _FP32_PEAK
    from paper_1708_03249_gb300 import hlb
    if _FP32_PEAK is None:
        _FP32_PEAK = (hlb.fp32_peak(False), hlb.fp32_peak(True))
    nominal = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    return max(_FP32_PEAK), {"measured_scalar_tflops": _FP32_PEAK[0], "measured_packed_tflops": _FP32_PEAK[1],
                              "nominal_tflops": nominal}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        sm.append(float(parts[1]))
                        mx = float(parts[2])
                    except ValueError:
                        continue
                    for name, val in zip(names, parts[5:9]):
                        if val.lower() == "active":
                            reasons.add(name)
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ------------------------------------------------------------------------------
def window_config(nx: int = 32, ny: int = 32) -> dict:
    """An nx x ny channel with the workload's velocity set, physics and cell
    size (so the same dt)."""
    cfg = dict(W.LARGE_2D)
    full_dx = cfg["Lx"] / cfg["nx"]
    cfg.update(nx=nx, ny=ny, Lx=nx * full_dx, Ly=ny * full_dx)
    return cfg


def oracle_sample(steps: int = 1, nx: int = 32, ny: int = 32, keep: bool = False):
    """Time the FP64 oracle on an nx x ny window of the same workload (same
    velocity set, physics and dt), ``steps`` RK-3 steps; returns (nv/s, secs,
    desc, cores) and, with keep, also (initial state, final moments)."""
    from oracle.solver import Solver, config_from
    cfg = window_config(nx, ny)
    s = Solver(config_from(cfg))
    s.init_equilibrium(1.0, 0.05, -0.02, 1.2)
    s.f *= W.perturbation(s.f.shape, seed=3, amplitude=0.02)
    f0 = s.f.copy() if keep else None
    t0, c0 = time.perf_counter(), time.process_time()
    s.step(steps)
    dt, cpu = time.perf_counter() - t0, time.process_time() - c0
    nv = nx * ny * s.vs.V * steps
    desc = f"{nx}x{ny} nodes of the workload's velocity set x {steps} RK-3 step(s), FP64 numpy oracle"
    out = (nv / dt, dt, desc, max(1, round(cpu / dt)))
    if keep:
        n, u, T, q = s.moments()
        out = out + (f0, (n.reshape(-1), u.reshape(-1, 3), T.reshape(-1), q.reshape(-1)))
    return out


_POOL_SOLVER = None


def _pool_init(cfg, seed):
    """Worker set-up (untimed): the oracle's tables and one problem's initial state."""
    global _POOL_SOLVER
    from oracle.solver import Solver, config_from
    s = Solver(config_from(cfg))
    s.init_equilibrium(1.0, 0.05, -0.02, 1.2)
    s.f *= W.perturbation(s.f.shape, seed=seed, amplitude=0.02)
    _POOL_SOLVER = s


def _pool_steps(steps):
    t0, c0 = time.perf_counter(), time.process_time()
    _POOL_SOLVER.step(steps)
    return time.perf_counter() - t0, time.process_time() - c0


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


class OraclePool:
    """The FP64 oracle on every host core: one spawned process per core, each
    advancing its own problem (by default an nx x ny window of the large
    channel: same velocity set, physics and dt, its own seeded perturbation;
    or the given configs, one per core), all at once.  The oracle's
    arithmetic is unchanged: the problems are independent, so the host's
    throughput is their node-velocity updates over the slowest one's wall
    time.  BLAS threads are pinned to one per process."""

    def __init__(self, workers: int = 0, nx: int = 32, ny: int = 32, cfgs=None, what: str = ""):
        import multiprocessing as mp
        self.workers = workers or (os.cpu_count() or 1)
        self.nx, self.ny = nx, ny
        self.cfgs = list(cfgs[: self.workers]) if cfgs else [window_config(nx, ny)] * self.workers
        self.workers = len(self.cfgs)
        self.what = what or f"independent {nx}x{ny}-node windows of the workload's velocity set"
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        ctx = mp.get_context("spawn")
        self.pools = [ctx.Pool(1, initializer=_pool_init, initargs=(c, 100 + r)) for r, c in enumerate(self.cfgs)]
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        for p in self.pools:                 # wait for every worker's set-up
            p.apply(time.sleep, (0,))
        self.V = None

    def run(self, steps: int):
        """(node-velocity updates/s over all workers, wall seconds, CPU seconds)."""
        t0 = time.perf_counter()
        res = [p.apply_async(_pool_steps, (steps,)) for p in self.pools]
        out = [r.get() for r in res]
        wall = time.perf_counter() - t0
        if self.V is None:
            from oracle.model import VelocitySet
            self.V = sum(c["nx"] * c["ny"] * VelocitySet(c["Qx"], c["Qy"], c["Qz"]).V for c in self.cfgs)
        nv = self.V * steps
        return nv / wall, wall, sum(o[1] for o in out)

    def describe(self, steps: int) -> str:
        return (f"{self.workers} {self.what} (one spawned process per host core, os.cpu_count() = "
                f"{os.cpu_count()}, CPU: {cpu_model()}) x {steps} RK-3 step(s) each, FP64 numpy oracle")

    def close(self):
        for p in self.pools:
            p.terminate()


def moment_errors(mom, ref) -> dict:
    """L-infinity error of each moment against the FP64 oracle, relative to
    max(max |M_ref|, s_M) with s_n = max n, s_u = sqrt(max T), s_T = max T,
    s_q = max n (max T)^(3/2)."""
    import numpy as np
    n, u, T, q = (np.asarray(a, dtype=np.float64) for a in mom)
    rn, ru, rT, rq = (np.asarray(a, dtype=np.float64) for a in ref)
    u, ru = u.reshape(-1, 3), ru.reshape(-1, 3)
    sT = np.abs(rT).max()
    return {"n": float(np.abs(n - rn).max() / np.abs(rn).max()),
            "u": float(np.abs(u - ru).max() / max(np.abs(ru).max(), math.sqrt(sT))),
            "T": float(np.abs(T - rT).max() / sT),
            "q": float(np.abs(q - rq).max() / max(np.abs(rq).max(), np.abs(rn).max() * sT ** 1.5))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    total_nv, total_t = 0.0, 0.0
    pool = OraclePool()
    desc = pool.describe(1) + " per timed step"
    cores = pool.workers
    for i in range(args.warmup + args.steps):
        rate, secs, _ = pool.run(1)
        if i >= args.warmup:
            total_nv += rate * secs
            total_t += secs
    pool.close()
    value = total_nv / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "node-velocity updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_t / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": desc},
        "cpu_baseline": {"value": value, "unit": "node-velocity updates/s", "cores": cores,
                         "kind": "oracle", "sample": desc, "cpu_model": cpu_model(),
                         "os_cpu_count": os.cpu_count()},
        "e2e": {"value": value, "unit": "node-velocity updates/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """The largest x over all ranks (the job's time is its slowest rank's);
    x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each did units_per_rank
    units in at most `seconds` (max over ranks)."""
    return world * units_per_rank / seconds


def roofline_of(hbm_achieved, hbm_peak, peak_kind, alu_achieved, alu_peak, sm_mhz, traffic, stage_avg_ms, kt,
                flop_nv):
    """Both roofs of the stage kernel; the binding one (the larger fraction)
    fills the top-level keys."""
    hbm = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
           "frac": hbm_achieved / hbm_peak, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
           "per_unit": BYTES_PER_NV_STAGE, "per_unit_desc": "algorithmic bytes per node-velocity per stage launch"}
    alu_meas, alu_ctx = fp32_alu_peak(sm_mhz)
    alu = {"bound": "alu", "achieved": alu_achieved, "peak": alu_meas, "unit": "TFLOP/s",
           "frac": alu_achieved / alu_meas,
           "peak_source": "measured: FP32 FMA chains on every SM (hlb_fp32_peak, the larger of scalar and packed)",
           "peak_context": alu_ctx, "frac_of_nominal": alu_achieved / alu_peak,
           "per_unit": flop_nv, "per_unit_desc": "algorithmic flops per node-velocity per stage launch"}
    top = dict(alu if alu["frac"] >= hbm["frac"] else hbm)
    top.update({"traffic": traffic, "kernel": "march_pair_kernel<WENO5, 16, 8>", "stage_avg_ms": stage_avg_ms,
                "stage_share": kt["stage_ms"] / max(kt["stage_ms"] + kt["wall_ms"], 1e-9),
                "hbm": hbm, "alu": alu})
    return top


# ------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    from paper_1708_03249_gb300 import build as hbuild
    from paper_1708_03249_gb300 import hlb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the oracle's host-core pool (rank 0 at N = 1 only), spawned before any CUDA call
    pool = OraclePool() if rank == 0 and world == 1 else None
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if not os.path.exists(hlb.LIB_PATH):
        if rank == 0:
            hbuild.build()
        if dist is not None:
            dist.barrier()
    stream = torch.cuda.Stream()
    cfg = with_precision(W.LARGE_2D, args.precision)
    workload = WORKLOAD if args.precision == "fp32" else f"{WORKLOAD}_{args.precision}"
    if args.nx or args.ny:        # a smaller grid of the same workload (profiling captures)
        nx = args.nx or cfg["nx"]
        ny = args.ny or cfg["ny"]
        cfg = W.scaled(cfg, nx=nx, ny=ny, Ly=cfg["Ly"] * ny / cfg["ny"], Lx=cfg["Lx"] * nx / cfg["nx"])
        workload = f"{WORKLOAD}_grid{nx}x{ny}"
    h = hlb.Handle(cfg, stream=stream.cuda_stream)
    nodes, values, state_bytes = h.nodes, h.values, h.state_bytes
    force_form = h.force_form(0)
    V = values // nodes
    h.init_equilibrium(1.0, 0.0, 0.0, 1.0)
    segments = h.autotune()              # marching-kernel segment length, timed per group (untimed here)

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up (graph replay off: the timed region launches eagerly with per-launch events)
    h.set_options(use_graphs=False, time_kernels=True)
    h.step(args.warmup)
    torch.cuda.synchronize()
    h.kernel_times(reset=True)
    h.launch_count(reset=True)

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("bench_timed")       # profilers: --nvtx --nvtx-include bench_timed/
        e0.record(stream)
        h.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier()
    ms = e0.elapsed_time(e1)
    kt = h.kernel_times(reset=True)
    launches = h.launch_count(reset=True)
    ms = max_over_ranks(ms, dist, "cuda")
    n, u, T, q = h.moments()
    finite = bool(np.isfinite(n).all() and np.isfinite(T).all())
    value = job_rate(nodes * V * args.steps, world, ms * 1e-3)

    # end to end through the C ABI with host buffers, every step: the state
    # uploaded from pinned memory, one RK-3 step, the moments read back into
    # pinned arrays.  Overlapped form (the e2e value): the upload of step k+1's
    # state is staged (hlb_prefetch_state, its own copy stream) while step k
    # runs, then committed; the first upload is inside the timed region.
    # Serial form (context): hlb_set_state, step, hlb_moments.
    pinned = torch.empty(values, dtype=torch.float32, pin_memory=True)
    h.get_state(pinned.numpy())
    h.set_options(use_graphs=True, time_kernels=False)
    e2e_iters = max(2, min(args.steps, 20))
    # page-locked result arrays, like the input: the moments land by DMA
    moms = [torch.empty(k * nodes, dtype=torch.float64, pin_memory=True).numpy() for k in (1, 3, 1, 1)]
    import ctypes
    ptrs = [m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for m in moms]
    lib = hlb.lib()

    def e2e_overlapped(iters):
        h.prefetch_state(pinned.data_ptr(), state_bytes)
        for it in range(iters):
            h.commit_state()
            if it + 1 < iters:
                h.prefetch_state(pinned.data_ptr(), state_bytes)
            h.step(1)
            hlb._check(lib.hlb_moments_async(h._h, *ptrs))      # read back while the next step runs
        hlb._check(lib.hlb_moments_wait(h._h))

    def e2e_serial(iters):
        for it in range(iters):
            hlb._check(lib.hlb_set_state(h._h, pinned.data_ptr(), state_bytes))
            h.step(1)
            hlb._check(lib.hlb_moments(h._h, *ptrs))

    def timed(fn):
        fn(1)                                    # untimed: staging buffer, graph
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn(e2e_iters)
        return max_over_ranks(time.perf_counter() - t0, dist, "cuda")

    e2e_value = job_rate(nodes * V * e2e_iters, world, timed(e2e_overlapped))
    e2e_serial_value = job_rate(nodes * V * e2e_iters, world, timed(e2e_serial))
    h.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peaks()
    stage_avg_ms = kt["stage_ms"] / max(kt["stage_launches"], 1)
    achieved = nodes * V * BYTES_PER_NV_STAGE / (stage_avg_ms * 1e-3) / 1e9
    flop_nv = flops_per_nv_stage(cfg)
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_max_mhz") or MAX_SM_MHZ
    alu_peak = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    alu_achieved = nodes * V * flop_nv / (stage_avg_ms * 1e-3) / 1e12
    traffic = None
    if os.path.exists(PROFILE_TRAFFIC):
        with open(PROFILE_TRAFFIC) as fh:
            prof = json.load(fh)
        if prof.get("kernel_hash") == kernel_source_hash():
            traffic = prof.get("dram_bytes_per_launch")
    # the same window on the GPU from the oracle's own initial state: the L-inf
    # moment errors of the timed kernels against the FP64 oracle
    _, _, _, _, f0_win, mom_ref = oracle_sample(steps=3, keep=True)
    cpu_baseline = None
    if pool is not None:
        cpu_rate, _, cpu_sec = pool.run(3)
        cpu_baseline = {"value": cpu_rate, "unit": "node-velocity updates/s", "cores": pool.workers,
                        "kind": "oracle", "sample": pool.describe(3), "cpu_model": cpu_model(),
                        "os_cpu_count": os.cpu_count(), "cpu_seconds": cpu_sec}
        pool.close()
    with hlb.Handle(with_precision(window_config(), args.precision), stream=stream.cuda_stream) as hw:
        hw.set_state(f0_win.reshape(-1).astype(np.float32))
        hw.step(3)
        errs = moment_errors(hw.moments(), mom_ref)
    line = {
        "metric": METRIC, "value": value, "unit": "node-velocity updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload, "nx": cfg["nx"], "ny": cfg["ny"], "velocities": V,
                   "nodes": nodes, "values_per_copy": values, "precision": "fp32",
                   "advection": "weno5", "parallelism": f"replicas{world}",
                   "l2": f"state ({state_bytes / 1e9:.2f} GB per copy) larger than L2; no flush needed",
                   "moments_finite": finite, "segment_cells": segments,
                   "force_term": FORCE_FORMS[force_form]},
        "roofline": roofline_of(achieved, peak, peak_kind, alu_achieved, alu_peak, sm_mhz, traffic,
                                stage_avg_ms, kt, flop_nv),
        "cpu_baseline": cpu_baseline,
        "accuracy": {"moment_linf_rel_err": errs, "bound": 1e-5, "within_bound": max(errs.values()) <= 1e-5,
                     "case": "the cpu_baseline window (32x32 nodes, 3 RK-3 steps) from the oracle's initial "
                             "state, FP32 kernels vs the FP64 oracle"},
        "e2e": {"value": e2e_value, "unit": "node-velocity updates/s",
                "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": 6 * 8 * nodes,
                "steps": e2e_iters,
                "form": "per step: the state from pinned memory (staged by hlb_prefetch_state on a copy "
                        "stream during the previous step, then hlb_commit_state), one RK-3 step, its "
                        "moments into pinned arrays (hlb_moments_async, landing while the next step runs; "
                        "hlb_moments_wait after the last); the first upload inside the timed region",
                "serial": e2e_serial_value},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------
# batched channels: one handle for all instances (FP32) vs per-instance FP64
# ------------------------------------------------------------------------------
def run_batched(args):
    """4096 independent 1D channels (SplitMix64 draws) advanced together in
    FP32 (one handle; each velocity-set group on the persistent kernel or the
    per-stage launches, whichever hlb_autotune measured faster), against the
    plain per-instance FP64 solve on the same GPU (a sample of instances, each
    its own FP64 handle stepped on its own)."""
    import ctypes

    import numpy as np
    import torch

    from paper_1708_03249_gb300 import build as hbuild
    from paper_1708_03249_gb300 import hlb

    insts = with_precision(W.batched_instances(args.ninst), args.precision)
    if args.qx:                       # one velocity-set group of the batch
        insts = [c for c in insts if c["Qx"] == args.qx]
    # the oracle's host-core pool (spawned before any CUDA call): the first
    # seeded instances of the batch, one per core
    pool = OraclePool(cfgs=insts, what="seeded batched channel instances (the batch's first ones)")
    torch.cuda.set_device(0)
    if not os.path.exists(hlb.LIB_PATH):
        hbuild.build()
    stream = torch.cuda.Stream()
    h = hlb.Handle(insts, stream=stream.cuda_stream)
    h.init_equilibrium()
    segments = h.autotune() if args.tune else None     # untuned: the persistent kernel where eligible
    groups = {}
    for i, c in enumerate(insts):
        key = (c["Qx"], c["Qy"])
        if key not in groups:
            f = h.step_form(i)
            groups[key] = {"velocities": 2 * c["Qx"] * max(c["Qy"], 1), "instances": 0, "values": 0,
                           "persistent": f["persistent"], "segment_cells": f["segment_cells"], "ctas": f["ctas"],
                           "tuned_step_ms": {"persistent": f["tuned_ms"][0], "per_stage": f["tuned_ms"][1]}}
        groups[key]["instances"] += 1
        groups[key]["values"] += c["nx"] * c["ny"] * groups[key]["velocities"]
    h.set_options(use_graphs=True, time_kernels=False)
    h.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.launch_count(reset=True)
    with ClockSampler(0) as clk:
        torch.cuda.nvtx.range_push("bench_timed")
        e0.record(stream)
        h.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    launches = h.launch_count(reset=True)
    nv = h.values
    nodes, state_bytes = h.nodes, h.state_bytes
    rate32 = nv * args.steps / (ms * 1e-3)
    n, u, T, q = h.moments()
    finite = bool(np.isfinite(n).all() and np.isfinite(T).all())
    # the stage kernels alone: per-stage launches with CUDA events (3 steps)
    h.set_options(use_graphs=False, time_kernels=True)
    h.kernel_times(reset=True)
    h.step(3)
    torch.cuda.synchronize()
    kt = h.kernel_times(reset=True)
    h.set_options(use_graphs=True, time_kernels=False)
    stage_ms_per_step = kt["stage_ms"] / 3.0
    # end to end through the C ABI with host buffers: per step the state from
    # pinned memory (staged during the previous step), one step, the moments
    # read back into pinned arrays while the next step runs
    pinned = torch.empty(nv, dtype=torch.float32, pin_memory=True)
    h.get_state(pinned.numpy())
    moms = [torch.empty(k * nodes, dtype=torch.float64, pin_memory=True).numpy() for k in (1, 3, 1, 1)]
    ptrs = [m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for m in moms]
    lib = hlb.lib()
    e2e_iters = max(2, min(args.steps, 20))

    def e2e(iters):
        h.prefetch_state(pinned.data_ptr(), state_bytes)
        for it in range(iters):
            h.commit_state()
            if it + 1 < iters:
                h.prefetch_state(pinned.data_ptr(), state_bytes)
            h.step(1)
            hlb._check(lib.hlb_moments_async(h._h, *ptrs))
        hlb._check(lib.hlb_moments_wait(h._h))

    e2e(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e(e2e_iters)
    e2e_value = nv * e2e_iters / (time.perf_counter() - t0)
    h.close()
    # accuracy: eight short seeded instances of the batch (all three velocity
    # sets) on the FP32 path against the FP64 oracle from the same state
    from oracle.solver import Solver, config_from
    acc_cfgs = [c for c in insts[:64] if c["nx"] <= 120][:8]
    with hlb.Handle(acc_cfgs, stream=stream.cuda_stream) as ha:
        ha.init_equilibrium(1.0, 0.05, 0.0, 1.1)
        f0 = ha.get_state().astype(np.float64) * W.perturbation(ha.values, seed=51, amplitude=0.05)
        ha.set_state(f0)
        f0 = ha.get_state().astype(np.float64)
        acc_steps = 20
        ha.step(acc_steps)
        mom = ha.moments()
    refs, off = [], 0
    for c in acc_cfgs:
        sv = Solver(config_from(c))
        sv.f = f0[off:off + sv.f.size].reshape(sv.f.shape).copy()
        off += sv.f.size
        sv.step(acc_steps)
        refs.append(sv.moments())
    ref = tuple(np.concatenate([r[k].reshape(-1, 3) if k == 1 else r[k].reshape(-1) for r in refs]) for k in range(4))
    errs = moment_errors(mom, ref)
    # per-instance FP64 solves of a sample (every ninst/fp64_sample-th instance)
    sample = insts[:: max(1, len(insts) // args.fp64_sample)][: args.fp64_sample]
    total_nv, total_ms = 0, 0.0
    for c in sample:
        c64 = dict(c, precision=W.FP64)
        hh = hlb.Handle(c64, stream=stream.cuda_stream)
        hh.init_equilibrium()
        hh.step(args.warmup)
        torch.cuda.synchronize()
        e0.record(stream)
        hh.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        total_nv += hh.values * args.steps
        hh.close()
    rate64 = total_nv / (total_ms * 1e-3)
    # roofline of the stage kernels (per-stage launches: the FP32 marching
    # kernels of every group, timed per launch)
    peak, peak_kind = measured_peaks()
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_max_mhz") or MAX_SM_MHZ
    hbm_ach = nv * BYTES_PER_NV_STAGE * 3 / (stage_ms_per_step * 1e-3) / 1e9
    flops = sum(g["values"] * flops_per_nv_stage(dict(Qx=qx, Qy=qy, ny=1, advection=W.WENO5, x_basis=W.X_HALF))
                for (qx, qy), g in groups.items())
    alu_peak, alu_ctx = fp32_alu_peak(sm_mhz)
    alu_ach = flops * 3 / (stage_ms_per_step * 1e-3) / 1e12
    hbm = {"bound": "hbm", "achieved": hbm_ach, "peak": peak, "unit": "GB/s", "frac": hbm_ach / peak,
           "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})", "per_unit": BYTES_PER_NV_STAGE}
    alu = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_ach / alu_peak,
           "peak_source": "measured: FP32 FMA chains on every SM (hlb_fp32_peak)", "peak_context": alu_ctx}
    roof = dict(alu if alu["frac"] >= hbm["frac"] else hbm)
    roof.update({"traffic": None, "kernel": "the groups' FP32 marching kernels (march1_kernel), per-stage launches",
                 "stage_ms_per_step": stage_ms_per_step, "hbm": hbm, "alu": alu})
    cpu_rate, _, cpu_sec = pool.run(3)
    cpu_baseline = {"value": cpu_rate, "unit": "node-velocity updates/s", "cores": pool.workers, "kind": "oracle",
                    "sample": pool.describe(3), "cpu_model": cpu_model(), "os_cpu_count": os.cpu_count(),
                    "cpu_seconds": cpu_sec}
    pool.close()
    line = {"metric": METRIC, "value": rate32, "unit": "node-velocity updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"batched_{args.ninst}_channels_splitmix64_seed{W.BATCH_SEED}",
                       "values_per_copy": nv, "moments_finite": finite, "segment_cells": segments,
                       "l2": f"state ({state_bytes / 1e9:.2f} GB per copy) larger than L2; no flush needed",
                       "groups": {f"{qx * 2}x{qy}": g for (qx, qy), g in groups.items()}},
            "roofline": roof,
            "cpu_baseline": cpu_baseline,
            "accuracy": {"moment_linf_rel_err": errs, "bound": 1e-5, "within_bound": max(errs.values()) <= 1e-5,
                         "case": f"{len(acc_cfgs)} short seeded instances of the batch, {acc_steps} RK-3 steps, "
                                 "FP32 kernels vs the FP64 oracle from the same state"},
            "e2e": {"value": e2e_value, "unit": "node-velocity updates/s", "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": 6 * 8 * nodes, "steps": e2e_iters,
                    "form": "per step: the state from pinned memory (hlb_prefetch_state during the previous step, "
                            "hlb_commit_state), one RK-3 step, the moments into pinned arrays (hlb_moments_async)"},
            "gpu_launches": launches,
            "clocks": clocks,
            "fp64_per_instance": {"value": rate64, "unit": "node-velocity updates/s",
                                  "instances": len(sample), "dtype": "f64",
                                  "desc": "each sampled instance its own FP64 handle, stepped alone"},
            "batched_fp32_over_fp64_per_instance": rate32 / rate64}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------
# the other configurations: one handle, graph replay, CUDA-event timing
# ------------------------------------------------------------------------------
OTHER_WORKLOADS = {
    "fp64_channel": ("1D FP64 channel, 64 cells, Qx=4 x Qy=4, upwind2, Kn=0.1, g=0.1 normal",
                     lambda: W.CHANNEL_1D_FP64),
    "stretched_channel": ("1D FP32 channel, 512 cells tanh A=0.9, Qx=8 x Qy=8, WENO5, Kn=0.1, g=0.5 at 30 deg",
                          lambda: W.channel_1d_stretched(0.1)),
    "box2d": ("2D FP32 box 256x256, Qx=16 x Qy=16, WENO5, Kn=0.05, g=0.2 at 45 deg", lambda: W.BOX_2D),
    "large2d_upwind2": ("the large 2D channel (1024x512, 16x8x8 velocities, FP32) with 2nd-order upwind "
                        "advection instead of WENO5", lambda: W.scaled(W.LARGE_2D, advection=W.UPWIND2)),
    "long_channel_q16": ("1D FP32 channel, 131072 cells, Qx=16 x Qy=16 (the batched set's largest slab, "
                         "tensor-core force term), WENO5, Kn=0.1, g=0.36 at 34 deg; 268 MB per copy",
                         lambda: W.make(Qx=16, Qy=16, nx=131072, T_left=1.0, T_right=1.5, ax=-0.3, ay=-0.2,
                                        Kn=0.1, advection=W.WENO5, precision=W.FP32)),
    "hhlb_20_200": ("the paper's ballistic runs (Sec. V) with its HHLB(20;200) model: 400 velocities, 24 cells "
                    "(A = 0.99), dt = 1e-4, WENO5, FP64, no collisions; the eight (g, Delta T) cases of its figure "
                    "as one handle", lambda: W.HHLB_BALLISTIC_SET),
    "hhlb_20_200_single": ("one case of the paper's ballistic runs (g = 1, Delta T = -0.4) with HHLB(20;200): "
                           "400 velocities x 24 cells, FP64", lambda: W.hhlb_ballistic(1.0, -0.4)),
}


def run_other(args):
    import numpy as np
    import torch

    from paper_1708_03249_gb300 import build as hbuild
    from paper_1708_03249_gb300 import hlb

    torch.cuda.set_device(0)
    if not os.path.exists(hlb.LIB_PATH):
        hbuild.build()
    desc, make_cfg = OTHER_WORKLOADS[args.workload]
    cfgs = with_precision(make_cfg(), args.precision)
    cfg = cfgs[0] if isinstance(cfgs, list) else cfgs
    stream = torch.cuda.Stream()
    with hlb.Handle(cfgs, stream=stream.cuda_stream) as h:
        h.init_equilibrium()
        segments = h.autotune()
        force_form = h.force_form(0)
        h.set_options(use_graphs=True, time_kernels=False)
        h.step(max(args.warmup, 30))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = max(args.steps, 30)
        torch.cuda.nvtx.range_push("bench_timed")
        e0.record(stream)
        h.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = e0.elapsed_time(e1)
        n, u, T, q = h.moments()
        nv = h.values
        # the stage kernels alone (CUDA events around each stage launch, 3 steps)
        h.set_options(use_graphs=False, time_kernels=True)
        h.kernel_times(reset=True)
        h.step(3)
        torch.cuda.synchronize()
        kt = h.kernel_times(reset=True)
    stage_ms = kt["stage_ms"] / max(kt["stage_launches"], 1)
    bytes_nv = BYTES_PER_NV_STAGE * (2 if cfg["precision"] == W.FP64 else 1)
    peak, peak_kind = measured_peaks()
    hbm = nv * bytes_nv / (stage_ms * 1e-3) / 1e9
    alu = nv * flops_per_nv_stage(cfg) / (stage_ms * 1e-3) / 1e12
    alu_peak, _ = fp32_alu_peak(MAX_SM_MHZ)
    stage = {"stage_avg_ms": stage_ms, "hbm_gbs": hbm, "hbm_frac": hbm / peak, "hbm_peak_source": peak_kind,
             "alu_tflops": alu, "alu_frac": alu / alu_peak, "alu_peak_tflops_measured": alu_peak,
             "per_unit_bytes": bytes_nv, "per_unit_flops": flops_per_nv_stage(cfg)}
    if cfg["precision"] == W.FP64:
        stage.update({"fp64_tflops": alu, "fp64_frac": alu / FP64_NOMINAL_TFLOPS,
                      "fp64_peak_source": "nominal 1.25 TFLOP/s"})
    line = {"metric": METRIC, "value": nv * steps / (ms * 1e-3), "unit": "node-velocity updates/s", "n_gpus": 1,
            "steps": steps, "warmup": max(args.warmup, 30), "ms_per_step": ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if cfg["precision"] == W.FP64 else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc, "values_per_copy": nv, "segment_cells": segments,
                       "force_term": FORCE_FORMS[force_form],
                       "moments_finite": bool(np.isfinite(n).all() and np.isfinite(T).all())},
            "stage_kernel": stage}
    print(json.dumps(line), flush=True)


def run_steady(args):
    """The stretched channel (512 cells, Q = 8 x 8, WENO5) toward its steady state:
    the FP64 path and the FP32 path with round-to-nearest and with stochastic
    stage outputs (hlb_set_rounding), from the same FP32-rounded perturbed
    equilibrium, stepped side by side in chunks, recording the last step's
    residual max|f^{n+1} - f^n| / (dt max f) of each and the largest relative
    deviation of each FP32 run's moments n, T, q from the FP64 ones.  A
    diagnostic of how far the FP32 state can follow the FP64 one over long
    runs, not a parity test."""
    import numpy as np
    import torch

    from paper_1708_03249_gb300 import build as hbuild
    from paper_1708_03249_gb300 import hlb

    torch.cuda.set_device(0)
    if not os.path.exists(hlb.LIB_PATH):
        hbuild.build()
    stream = torch.cuda.Stream()
    chunk = 20000
    total = max(chunk, args.steps if args.steps > 20 else 220000)
    per_kn = {}
    t0 = time.perf_counter()
    for Kn in W.CHANNEL_1D_STRETCHED_KN:
        c32, c64 = W.channel_1d_stretched(Kn), W.channel_1d_stretched(Kn, precision=W.FP64)
        with hlb.Handle(c64, stream=stream.cuda_stream) as h, hlb.Handle(c32, stream=stream.cuda_stream) as g, \
                hlb.Handle(c32, stream=stream.cuda_stream) as gs:
            g.init_equilibrium(1.0, 0.0, 0.0, 1.0)
            f0 = (g.get_state().astype(np.float64) * W.perturbation(g.values, seed=1, amplitude=0.05)).astype(np.float32)
            g.set_state(f0)
            gs.set_state(f0)
            gs.set_rounding(True)
            h.set_state(f0.astype(np.float64))
            hist, steps = [], 0

            def dev(a, b):
                return float(max(np.abs(a[0] - b[0]).max() / np.abs(b[0]).max(),
                                 np.abs(a[2] - b[2]).max() / np.abs(b[2]).max(),
                                 np.abs(a[3] - b[3]).max() / max(np.abs(b[3]).max(), 1e-300)))
            while steps < total:
                for hh in (h, g, gs):
                    hh.step(chunk)
                steps += chunk
                m64 = h.moments()
                hist.append({"steps": steps, "residual_fp64": float(h.diag()[1][0]),
                             "residual_fp32": float(g.diag()[1][0]), "residual_fp32_sr": float(gs.diag()[1][0]),
                             "moment_dev": dev(g.moments(), m64), "moment_dev_sr": dev(gs.moments(), m64)})
            per_kn[f"{Kn:g}"] = {"dt": h.dt(), "history": hist}
    line = {"metric": "steady-state residual and FP32 moment deviation from FP64", "n_gpus": 1,
            "config": {"workload": "stretched_channel_steady_state",
                       "desc": "1D channel, 512 cells tanh A=0.9, Qx=8 x Qy=8, WENO5, T 0.5/1.5, g=0.5 at 30 deg; "
                               "FP64 and FP32 paths side by side from one perturbed equilibrium",
                       "chunk_steps": chunk, "steps": total},
            "per_kn": per_kn, "seconds": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="large2d",
                    choices=["large2d", "batched", "stretched_steady_state"] + sorted(OTHER_WORKLOADS),
                    help="large2d: the JSON line of record; batched: the 4096-channel batch vs per-instance "
                         "FP64; stretched_steady_state: FP32 and FP64 stretched channels stepped side by side "
                         "toward the steady state (--steps: total steps, default 220000); the others time one "
                         "handle of that configuration")
    ap.add_argument("--ninst", type=int, default=4096)
    ap.add_argument("--nx", type=int, default=0, help="profiling: the large 2D workload on a smaller grid")
    ap.add_argument("--ny", type=int, default=0)
    ap.add_argument("--fp64-sample", type=int, default=64)
    ap.add_argument("--qx", type=int, default=0, help="batched: only the instances with this Qx (4, 8 or 16)")
    ap.add_argument("--tune", type=int, default=1, help="batched: 0 skips hlb_autotune (persistent kernel kept)")
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS),
                    help="FP32 workloads: the force term's form (fp32: the library's choice; tf32x3, bf16split: "
                         "on the tensor cores)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "stretched_steady_state":
        run_steady(args)
    elif args.workload in OTHER_WORKLOADS:
        run_other(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
