"""Write the oracle's long-run moments for the FP32 parity tests at length.

    python tests/golden/make_long_runs.py [--workers N] [--only PREFIX]

Calls only ``oracle/`` (and the seeded parameter sets of ``workloads.py``).
Each case starts from the oracle's own rest equilibrium (n = 1, u = 0, T = 1)
times the seeded factors 1 + 0.05 U(-1, 1), rounded to FP32 (so that the FP32
path can start from exactly the same state), runs the stated number of RK-3
steps in FP64 and stores, in ``tests/golden/long_runs/<case>.npz``:
n, u (nodes x 3), T, q per node in state order, the particle number N, the
residual max|f^{n+1} - f^n| / (dt max f) of the last step, and the config.

Cases (the oracle takes 2-5 ms per node and step at Q = 8 and 16, because its
half-range equilibrium falls back to 80-digit arithmetic wherever the FP64
rounding bound exceeds 1e-12, so the sizes below are what one host can run):
  stretched_kn*  the 512-cell stretched channel, Q = 8 x 8, at each Knudsen
                 number, 3000 steps (t = 0.176; the residual reached is stored);
  box24          the 2D box's velocity set and physics (Q = 16 x 16, walls 1 and
                 1.2, g = 0.2 at 45 deg, Kn = 0.05) on 24 x 24 cells, 2000 steps;
  large24        the large channel's velocity set and physics (16 x 8 x 8 velocities,
                 walls 1 and 2, a = (-0.3, -0.3, 0), Kn = 0.5, its cell size and time
                 step) on a 24 x 24-cell window, 500 steps (its stated length);
  batched_<i>    the first 64 seeded batched instances, 5000 steps each, except
                 the sixteen whose run would exceed 5000 s of one core here (Q = 16
                 with nx >= 258, Q = 8 with nx >= 452), which run 500 steps.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "long_runs")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1708_03249_gb300 import workloads as W  # noqa: E402

STRETCHED_STEPS = 3000
BOX_STEPS = 2000
BOX_N = 24
LARGE_STEPS = W.LARGE_2D_STEPS
LARGE_N = 24
BATCH_COUNT = 64
BATCH_LONG, BATCH_SHORT = W.BATCH_STEPS, 500
# measured one-core cost of the oracle, seconds per node and RK-3 step
_COST = {4: 0.18e-3, 8: 2.34e-3, 16: 5.32e-3}
_SHORT_ABOVE_S = 5000.0


def batch_steps(cfg: dict) -> int:
    est = cfg["nx"] * cfg["ny"] * BATCH_LONG * _COST[cfg["Qx"]]
    return BATCH_LONG if est <= _SHORT_ABOVE_S else BATCH_SHORT


def cases():
    """(name, config dict, steps, perturbation seed) for every case."""
    out = []
    for k, Kn in enumerate(W.CHANNEL_1D_STRETCHED_KN):
        out.append((f"stretched_kn{Kn:g}", W.channel_1d_stretched(Kn), STRETCHED_STEPS, 500 + k))
    out.append((f"box{BOX_N}", W.scaled(W.BOX_2D, nx=BOX_N, ny=BOX_N), BOX_STEPS, 600))
    out.append((f"large{LARGE_N}", large_window(), LARGE_STEPS, 700))
    for i, c in enumerate(W.batched_instances(BATCH_COUNT)):
        out.append((f"batched_{i:02d}", c, batch_steps(c), 1000 + i))
    return out


def large_window(n: int = LARGE_N) -> dict:
    """The large channel's workload on an n x n window: same velocity set,
    physics, cell size and time step (the channel is n cells wide)."""
    c = W.LARGE_2D
    return W.scaled(c, nx=n, ny=n, Lx=c["Lx"] * n / c["nx"], Ly=c["Ly"] * n / c["ny"])


def initial_state(cfg: dict, seed: int) -> np.ndarray:
    """Rest equilibrium of the oracle times the seeded factors, rounded to FP32."""
    from oracle.solver import Solver, config_from
    s = Solver(config_from(cfg))
    f = s.init_equilibrium()
    f = f * W.perturbation(f.shape, seed=seed)
    return f.astype(np.float32).astype(np.float64)


def run_case(task):
    name, cfg, steps, seed = task
    from oracle.solver import Solver, config_from
    t0 = time.time()
    s = Solver(config_from(cfg))
    s.f = initial_state(cfg, seed).reshape(s.f.shape)
    s.step(steps - 1)
    prev = s.f.copy()
    s.step(1)
    n, u, T, q = s.moments()
    np.savez_compressed(
        os.path.join(OUT, name + ".npz"),
        n=n.reshape(-1), u=u.reshape(-1, 3), T=T.reshape(-1), q=q.reshape(-1),
        N=s.total_number(), residual=s.residual(prev, s.f), steps=steps, seed=seed,
        dt=s.dt, config=json.dumps(cfg), seconds=time.time() - t0)
    return name, time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--only", default="")
    args = ap.parse_args()
    os.makedirs(OUT, exist_ok=True)
    todo = [c for c in cases() if c[0].startswith(args.only)
            and not os.path.exists(os.path.join(OUT, c[0] + ".npz"))]
    cost = lambda c: c[1]["nx"] * c[1]["ny"] * c[2] * _COST[c[1]["Qx"]]
    todo.sort(key=cost, reverse=True)          # longest first
    print(f"{len(todo)} cases, about {sum(map(cost, todo)):.0f} core-seconds", flush=True)
    with mp.get_context("spawn").Pool(args.workers) as pool:
        for name, sec in pool.imap_unordered(run_case, todo):
            print(f"{name}: {sec:.0f} s", flush=True)


if __name__ == "__main__":
    main()
