"""Write the stored oracle gradient of the film-solve workload (imports oracle/ and workloads.py only).

The workload (workloads.adjoint_film): a 512^2-cell square film in a 1024^2 grid, n = 30, a
lognormal jc map (sigma 0.2, seed 5), h_e through 16 knots on [0, T] with the baseline values
0.5 t / T.  The map has frozen decisions: N Bogacki-Shampine steps of [0, T]
(workloads.segment_steps: uniform inside each knot segment, none across a knot) from a zero
state, every right-hand side warm-started from the previous call (the first one cold), with the
outside-iteration counts that the stop test of Section 2.3 (2e-4) chose in a forward run of the
same steps with the oracle's FilmProblem (calls one after another, each from the previous call's
iterate).  Target: h_z(T) of the same frozen map with a second jc map (seed 6).
Loss L = 1/2 dx dy sum (h_z(T) - target)^2.

Stored (tests/golden/adjoint_<workload>.json): T, N, the counts, L, dL/d(knot values), dL/djc at
32 seeded random film cells, and the directional derivatives <dL/djc, d> for two seeded
directions d = jc * z (z ~ N(0,1) per cell), with the oracle's wall time.

  python tests/golden/make_adjoint_golden.py [--grid 1024] [--steps 400] [--T 0.1] [--ckpt 20]
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
from oracle.film2d import FilmProblem  # noqa: E402
from oracle.waveform import Waveform  # noqa: E402

CELL_SEED, DIR_SEEDS = 53, (54, 55)


def problem(wl, jc):
    return FilmProblem(wl.nx, wl.ny, wl.Lx, wl.Ly, wl.mask, n=wl.n, rho_out=wl.rho_out,
                       waveform=Waveform(*wl.he_knots), jc=jc, sigma=wl.sigma, lam=wl.lam,
                       iter_tol=wl.iter_tol, iter_max=wl.iter_max)


def stop_test_counts(wl, jc, steps):
    """The counts the stop test chooses along the frozen steps (calls one after another)."""
    p = problem(wl, jc)
    a = FilmAdjoint(p)
    kt, kv = np.array(wl.he_knots[0]), np.array(wl.he_knots[1])
    y = np.zeros((wl.ny, wl.nx))
    counts = []
    for t, h in steps:
        k = a._segment(kt, t, t + h)
        ks = []
        for aa, kprev in ((0.0, None), (0.5, 0), (0.75, 1)):
            gs = y if kprev is None else y + aa * h * ks[kprev]
            kj, it, st = p.rhs(t, gs, k)
            if st != 0:          # the cap was reached: the frozen map uses the cap as the count
                print(f"the stop test reached the cap ({it}) at t = {t}", flush=True)
            ks.append(kj)
            counts.append(int(it))
        y = y + h * (2.0 / 9.0 * ks[0] + 1.0 / 3.0 * ks[1] + 4.0 / 9.0 * ks[2])
    return counts


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--T", type=float, default=0.1)
    ap.add_argument("--ckpt", type=int, default=20)
    ap.add_argument("--iter-max", type=int, default=0, help="cap of the stop-test run (0: workload's)")
    args = ap.parse_args()
    wl = W.adjoint_film(args.grid, precision=0, T=args.T)
    if args.iter_max:
        wl.iter_max = args.iter_max
    jc = wl.jc_map
    jc6 = W.jc_map_lognormal((wl.ny, wl.nx), seed=6, sigma=0.2)
    kt, kv = wl.he_knots
    steps = W.segment_steps(kt, args.steps)
    w0 = time.time()
    counts = stop_test_counts(wl, jc, steps)
    print(f"counts: {len(counts)} calls, mean {np.mean(counts):.2f}, {time.time() - w0:.0f} s", flush=True)
    g0 = np.zeros((wl.ny, wl.nx))
    a6 = FilmAdjoint(problem(wl, jc6))
    y6 = a6.solve(g0, jc6, kt, kv, steps, counts)
    target = a6._he(np.array(kt), np.array(kv), args.T)[0] + a6.T(a6.p.Kh, y6)
    print(f"target: {time.time() - w0:.0f} s", flush=True)
    a = FilmAdjoint(problem(wl, jc))
    L, cb, vb, _ = a.gradient(g0, jc, kt, kv, steps, target, counts, ckpt_every=args.ckpt)
    wall = time.time() - w0
    film = np.argwhere(wl.mask == 1)
    cells = film[W.rng(CELL_SEED).choice(len(film), 32, replace=False)]
    dirs = [jc * W.rng(s).standard_normal(jc.shape) for s in DIR_SEEDS]
    out = {"workload": wl.name, "grid": [wl.nx, wl.ny], "T": args.T, "steps": args.steps,
           "iter_max": wl.iter_max,
           "ckpt_every": args.ckpt, "counts": counts, "loss": L, "knots_bar": vb.tolist(),
           "cells": cells.tolist(), "jcbar_cells": [float(cb[iy, ix]) for iy, ix in cells],
           "cell_seed": CELL_SEED, "direction_seeds": list(DIR_SEEDS),
           "directional": [float((cb * d).sum()) for d in dirs],
           "jcbar_abs_sum": float(np.abs(cb).sum()), "jcbar_l2": float(np.linalg.norm(cb)),
           "oracle_seconds": wall, "fft_workers": _fft.workers(),
           "made_by": "tests/golden/make_adjoint_golden.py (oracle/ only)"}
    path = os.path.join(HERE, f"adjoint_{wl.name}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(json.dumps({k: v for k, v in out.items() if k not in ("counts", "cells", "jcbar_cells")}))


if __name__ == "__main__":
    main()
