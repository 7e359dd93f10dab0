"""Write the stored oracle gradient of the film-solve workload (imports oracle/ and workloads.py only).

The workload (workloads.adjoint_film): a 512^2-cell square film in a 1024^2 grid, n = 30, a
lognormal jc map (sigma 0.2, seed 5), h_e through 16 knots on [0, T] with the baseline values
0.5 t / T.  The map has frozen decisions, taken from the oracle's own adaptive run of the
workload (Bogacki-Shampine with rtol = atol = 1e-6 and the stop test of Section 2.3, from a zero
state): its accepted steps (t, h) and, per step, the outside-iteration counts of k1 (that of
the previous step's k4 when k1 was reused), k2 and k3.  (Uniform steps of T/N are unstable for
this explicit scheme with n = 30 near the critical state, so the steps come from the adaptive
run; the same frozen steps are unstable for another jc map too.)  The frozen map warm-starts
every call from the previous one (the first one cold).
Target: h_z(T) of the oracle's own adaptive run (same tolerances and start) with a second jc map
(seed 6).  Loss L = 1/2 dx dy sum (h_z(T) - target)^2.

Stored (tests/golden/adjoint_<workload>.json): T, the steps, the counts, L, dL/d(knot values),
dL/djc at 32 seeded random film cells, and the directional derivatives <dL/djc, d> for two
seeded directions d = jc * z (z ~ N(0,1) per cell), with the oracle's wall time; and, so that a
user of the stored values can rebuild the target with an FP64 adaptive run of their own and
check it, the target run's attempt and acceptance counts and the target's norm, sum and values
at the 32 cells and at 32 seeded free-space cells.

  python tests/golden/make_adjoint_golden.py [--grid 1024] [--T 0.04] [--ckpt 20]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import _fft  # noqa: E402
from oracle.adjoint2d import FilmAdjoint  # noqa: E402
from oracle.bs23 import BS23  # noqa: E402
from oracle.film2d import FilmProblem  # noqa: E402
from oracle.waveform import Waveform  # noqa: E402

CELL_SEED, DIR_SEEDS, OUT_SEED = 53, (54, 55), 56


def problem(wl, jc):
    return FilmProblem(wl.nx, wl.ny, wl.Lx, wl.Ly, wl.mask, n=wl.n, rho_out=wl.rho_out,
                       waveform=Waveform(*wl.he_knots), jc=jc, sigma=wl.sigma, lam=wl.lam,
                       iter_tol=wl.iter_tol, iter_max=wl.iter_max)


def adaptive_run(wl, jc):
    """The oracle's adaptive run: (accepted steps, per-step counts (k1, k2, k3), attempts,
    h_z(T))."""
    p = problem(wl, jc)
    s = BS23(p.rhs, p.wf, rtol=wl.rtol, atol=wl.atol, on_accept=p.accept, on_attempt=p.begin_attempt)
    s.start(wl.t0, np.zeros((wl.ny, wl.nx)), wl.t1)
    if s.advance(wl.t1) != 0:
        raise SystemExit("the oracle's adaptive run stopped early")
    steps, counts, k4_prev = [], [], None
    for e in s.log:
        if e.outcome != 1:
            continue
        k1 = e.iters[0] if e.iters[0] >= 0 else k4_prev
        steps.append((e.t, e.h))
        counts += [int(k1), int(e.iters[1]), int(e.iters[2])]
        k4_prev = e.iters[3]
    return steps, counts, len(s.log), p.hz(wl.t1, s.y)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=1024)
    ap.add_argument("--T", type=float, default=0.04)
    ap.add_argument("--ckpt", type=int, default=20)
    args = ap.parse_args()
    wl = W.adjoint_film(args.grid, precision=0, T=args.T)
    jc = wl.jc_map
    jc6 = W.jc_map_lognormal((wl.ny, wl.nx), seed=6, sigma=0.2)
    kt, kv = wl.he_knots
    w0 = time.time()
    steps, counts, attempts, _ = adaptive_run(wl, jc)
    print(f"adaptive run: {len(steps)} accepted steps of {attempts} attempts, mean count "
          f"{np.mean(counts):.2f}, {time.time() - w0:.0f} s", flush=True)
    g0 = np.zeros((wl.ny, wl.nx))
    steps6, _, attempts6, target = adaptive_run(wl, jc6)
    print(f"target: {len(steps6)} accepted steps of {attempts6} attempts, {time.time() - w0:.0f} s",
          flush=True)
    a = FilmAdjoint(problem(wl, jc))
    L, cb, vb, _ = a.gradient(g0, jc, kt, kv, steps, target, counts, ckpt_every=args.ckpt)
    wall = time.time() - w0
    film = np.argwhere(wl.mask == 1)
    cells = film[W.rng(CELL_SEED).choice(len(film), 32, replace=False)]
    free = np.argwhere(wl.mask == 0)
    out_cells = free[W.rng(OUT_SEED).choice(len(free), 32, replace=False)]
    dirs = [jc * W.rng(s).standard_normal(jc.shape) for s in DIR_SEEDS]
    out = {"workload": wl.name, "grid": [wl.nx, wl.ny], "T": args.T, "n_steps": len(steps),
           "steps": [[float(t), float(h)] for t, h in steps], "adaptive_attempts": attempts,
           "rtol": wl.rtol, "atol": wl.atol,
           "ckpt_every": args.ckpt, "counts": counts, "loss": L, "knots_bar": vb.tolist(),
           "cells": cells.tolist(), "jcbar_cells": [float(cb[iy, ix]) for iy, ix in cells],
           "cell_seed": CELL_SEED, "direction_seeds": list(DIR_SEEDS),
           "directional": [float((cb * d).sum()) for d in dirs],
           "jcbar_abs_sum": float(np.abs(cb).sum()), "jcbar_l2": float(np.linalg.norm(cb)),
           "target_jc_seed": 6, "target_accepted": len(steps6), "target_attempts": attempts6,
           "target_l2": float(np.linalg.norm(target)), "target_sum": float(target.sum()),
           "target_cells": [float(target[iy, ix]) for iy, ix in cells],
           "out_cells": out_cells.tolist(),
           "target_out_cells": [float(target[iy, ix]) for iy, ix in out_cells],
           "oracle_seconds": wall, "fft_workers": _fft.workers(),
           "made_by": "tests/golden/make_adjoint_golden.py (oracle/ only)"}
    path = os.path.join(HERE, f"adjoint_{wl.name}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(json.dumps({k: v for k, v in out.items()
                      if k not in ("counts", "cells", "jcbar_cells", "steps", "out_cells", "target_cells",
                                   "target_out_cells")}))


if __name__ == "__main__":
    main()
