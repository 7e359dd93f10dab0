"""Write the stored reference ramps of the FP64 oracle (imports oracle/ and workloads.py only).

Each case integrates the oracle's right-hand side (Section 2.2 for the film, Section 3.1 for the
cube) with its Bogacki-Shampine 3(2) integrator, free running from a zero state at t0, and stores
readouts at fixed output times in tests/golden/<name>.npz, with the parameters, the integrator's
step counts and the wall time in a JSON sidecar.  The CUDA path's full-ramp tests compare their own
free-running ramps with these files at the precision form's tolerance (2e-4 relative L2).

  rect_film_2048   the 1024 x 512-cell rectangle in a 2048^2 grid, n = 30,
                   h_e = 0.8 sin(2 pi t): m_z at every output time, h_z on every 16th cell of
                   both axes at the snapshot times
  cube_128         the cube of 64^3 cells in a 128^3 grid, n = 25, rho_out = 5,
                   h_e,z ramped to 0.25 on [0, 0.5] and held: m at every output time, j on every
                   4th cell of the cube (and its one-cell rim) at the snapshot times

  python tests/golden/make_ramp_goldens.py <case> [--t-end T] [--n-out K]

--t-end stops the ramp early (a segment [t0, T] of the stated ramp); the sidecar records it.
The files are rewritten at every field snapshot, so an interrupted run leaves a shorter segment.
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
from oracle.bs23 import BS23  # noqa: E402
from oracle.bulk3d import BulkProblem  # noqa: E402
from oracle.film2d import FilmProblem  # noqa: E402
from oracle.waveform import Waveform  # noqa: E402

FILM_STRIDE = 16       # h_z samples: every 16th cell of each axis
CUBE_STRIDE = 4        # j samples: every 4th cell of each axis, over the cube and its rim


def _waveform(wl):
    if wl.he_knots is not None:
        return Waveform(*wl.he_knots)
    return Waveform(sin_amp=wl.he_sin[0], sin_period=wl.he_sin[1])


def film_case(t_end: float, n_out: int):
    wl = W.rect_film_2048(precision=0)
    o = FilmProblem(wl.nx, wl.ny, wl.Lx, wl.Ly, wl.mask, n=wl.n, rho_out=wl.rho_out,
                    waveform=_waveform(wl), jc=wl.jc, sigma=wl.sigma, lam=wl.lam,
                    iter_tol=wl.iter_tol, iter_max=wl.iter_max)
    s = BS23(o.rhs, o.wf, rtol=wl.rtol, atol=wl.atol, on_accept=o.accept, on_attempt=o.begin_attempt)
    y0 = np.zeros((wl.ny, wl.nx))
    readout = lambda t, y: (np.array([o.magnetization(y)]), o.hz(t, y)[::FILM_STRIDE, ::FILM_STRIDE])
    return wl, s, y0, readout


def cube_case(t_end: float, n_out: int):
    wl = W.cube_bulk(128, precision=0)
    o = BulkProblem(wl.nx, wl.ny, wl.nz, wl.Lx, wl.Ly, wl.Lz, wl.mask, n=wl.n, rho_out=wl.rho_out,
                    waveform=_waveform(wl), he_dir=wl.vector_he, jc=wl.jc, sigma=wl.sigma,
                    iter_tol=wl.iter_tol, iter_max=wl.iter_max)
    s = BS23(o.rhs, o.wf, rtol=wl.rtol, atol=wl.atol)
    y0 = np.zeros((3, wl.nz, wl.ny, wl.nx))
    lo, hi = wl.nx // 4 - 4, 3 * wl.nx // 4 + 4          # the cube (cells 32..95) and a rim

    def readout(t, y):
        j = o.current(y)[:, lo:hi:CUBE_STRIDE, lo:hi:CUBE_STRIDE, lo:hi:CUBE_STRIDE]
        return o.magnetization(y), j
    return wl, s, y0, readout


CASES = {"rect_film_2048": film_case, "cube_128": cube_case}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--t-end", type=float, default=1.0)
    ap.add_argument("--n-out", type=int, default=20)
    ap.add_argument("--snapshots", type=int, default=4, help="field snapshots, evenly spaced")
    args = ap.parse_args()
    wl, s, y0, readout = CASES[args.case](args.t_end, args.n_out)
    t0 = wl.t0
    t_out = t0 + (args.t_end - t0) * np.arange(1, args.n_out + 1) / args.n_out
    snap_every = max(1, args.n_out // args.snapshots)
    s.start(t0, y0, wl.t1)           # first step as the library chooses it for the stated ramp
    ms, fields, t_fields = [], [], []
    w0 = time.time()
    out = os.path.join(HERE, f"ramp_{wl.name}.npz")

    def save(n_done: int, wall: float):
        """Write what has been computed so far (the ramp up to output time n_done)."""
        np.savez_compressed(out, t_out=t_out[:n_done], m=np.array(ms), t_fields=np.array(t_fields),
                            fields=np.array(fields))
        meta = {"workload": wl.name, "case": args.case, "t0": t0, "t_end": float(t_out[n_done - 1]),
                "t_end_requested": args.t_end, "n_out": n_done, "field": "h_z" if wl.dim == 2 else "j",
                "field_stride": FILM_STRIDE if wl.dim == 2 else CUBE_STRIDE,
                "grid": [wl.nx, wl.ny, wl.nz], "n": wl.n, "rho_out": wl.rho_out,
                "rtol": wl.rtol, "atol": wl.atol, "iter_tol": wl.iter_tol,
                "attempts": len(s.log), "accepted": sum(1 for e in s.log if e.outcome == 1),
                "rhs_evals": int(sum(sum(1 for i in e.iters if i >= 0) for e in s.log)),
                "outside_iterations": int(sum(sum(i for i in e.iters if i > 0) for e in s.log)),
                "oracle_seconds": wall, "fft_workers": _fft.workers(),
                "made_by": "tests/golden/make_ramp_goldens.py (oracle/ only)"}
        with open(out.replace(".npz", ".json"), "w") as f:
            json.dump(meta, f, indent=1)
        return meta

    meta = None
    for k, t in enumerate(t_out):
        st = s.advance(float(t))
        if st != 0:
            raise SystemExit(f"oracle ramp stopped with status {st} at t = {s.t}")
        m, f = readout(float(t), s.y)
        ms.append(m)
        if (k + 1) % snap_every == 0 or k == len(t_out) - 1:
            fields.append(f)
            t_fields.append(float(t))
            meta = save(k + 1, time.time() - w0)     # a snapshot closes a stored segment
        acc = sum(1 for e in s.log if e.outcome == 1)
        print(f"t = {t:.4f}  steps {len(s.log)} ({acc} accepted)  {time.time() - w0:.0f} s", flush=True)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
