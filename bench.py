"""Benchmark: right-hand-side evaluations per second of the FFT method-of-lines film solver.

Workload: rectangular film 1024 x 512 cells (aspect 2:1) in a 2048 x 2048 periodic grid, n = 30,
h_e = 0.8 sin(2 pi t), FP32 transforms and power law with FP64 state (precision form).  One
benchmark step is one BS23 step attempt of the whole right-hand-side path (stage input,
smoothed gradient, power law, curl, warm-started outside iteration with its stop test, error
norm and step control), all in the persistent CUDA kernel.  The metric counts every
right-hand-side evaluation the steps performed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (under torch.distributed.run): every rank advances its own replica of the film (the film
does not shard); value = all ranks' evaluations / max time over ranks.
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
METRIC = "RHS evals/s"
UNIT = "RHS/s"


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    v = d[k]
                    return float(v["value"] if isinstance(v, dict) else v), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# the sources the persistent kernels are compiled from (host-only API code excluded)
KERNEL_SOURCES = ("mf_common.cuh", "mf_fft.cuh", "mf_passes.cuh", "mf_rhs_common.cuh",
                  "mf_tables.h", "mf_film.cuh", "mf_film.cu", "mf_film_batch.cu", "mf_bulk.cu")


def source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1801_04869_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per algorithmic byte from the committed ncu capture of this kernel, if it was
    taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    src = source_hash()
    for line in open(p):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == src and parts[1] == kernel and parts[2] == workload:
            return float(parts[3])
    return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mf_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def rhs_bytes(n_rhs: int, n_iters: int, M: float) -> float:
    """Algorithmic HBM bytes of the film right-hand side: (19 + 14 I) M per evaluation,
    M = bytes of one real field at transform precision, I = outside iterations."""
    return (19.0 * n_rhs + 14.0 * n_iters) * M


def _oracle_problem(wl):
    from oracle.film2d import FilmProblem
    from oracle.waveform import Waveform
    wf = Waveform(*wl.he_knots) if wl.he_knots else Waveform(sin_amp=wl.he_sin[0], sin_period=wl.he_sin[1])
    return FilmProblem(wl.nx, wl.ny, wl.Lx, wl.Ly, wl.mask, n=wl.n, rho_out=wl.rho_out, waveform=wf,
                       iter_tol=wl.iter_tol, iter_max=wl.iter_max, lam=wl.lam)


def bulk_leg(native, W, torch, steps: int = 6, warmup: int = 2, n_grid: int = 128, tune: bool = True,
             cufft: bool = True):
    """Secondary line: the 3D cube (n_grid/2 cells per side in n_grid^3), FP32 transforms,
    after mf_autotune has picked the work-item shape and launch width (reported beside it;
    tune=False keeps the size rules' choice).  The warm-up and the timed steps are one
    persistent launch each; with cufft, cuFFT's transform floor of one vector round trip on the
    same grid is timed afterwards beside the library's time per vector round trip."""
    wl = W.cube_bulk(n_grid, precision=1)
    p = native.from_workload(wl)
    tune = p.mf_autotune(reps=2, force_iters=2) if tune else None   # transform work does not depend on the values
    p.mf_set_state(0.0, None, h=1e-3)
    p.mf_advance(1.0, max_attempts=warmup)
    torch.cuda.synchronize()
    i0 = p.mf_get_info()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(p.stream)
    p.mf_advance(1.0, max_attempts=steps)
    e1.record(p.stream)
    torch.cuda.synchronize()
    i1 = p.mf_get_info()
    sec = e0.elapsed_time(e1) / 1000.0
    n_rhs, n_it = i1["n_rhs"] - i0["n_rhs"], i1["n_iters"] - i0["n_iters"]
    M3 = float(n_grid) ** 3 * 4.0
    alg = (60.0 * n_rhs + 60.0 * n_it) * M3
    peak, kind = hbm_peak()
    return {"workload": wl.name, "value": n_rhs / sec, "unit": UNIT, "steps": i1["n_attempts"] - i0["n_attempts"],
            "mean_outside_iterations": n_it / max(n_rhs, 1),
            "roofline": {"bound": "hbm", "achieved": alg / sec / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / sec / 1e9 / peak, "peak_kind": kind,
                         "bytes_model": f"(60 + 60 I) M3 per RHS, M3 = {n_grid}^3 x 4 B"},
            "ms_per_vector_round_trip": 1000.0 * sec / (2 * n_rhs + 2 * n_it),
            "cufft": cufft3_leg(torch, n_grid) if cufft else None,
            "autotune": tune}


def autotune_leg(native, W, torch, n_grid: int):
    """Secondary line: mf_autotune on the benchmark film (a separate problem object): the
    work-item shapes and launch widths it timed and the one it keeps, against the size rules'
    choice that the timed region uses."""
    wl = W.rect_film_2048(precision=1, n_grid=n_grid)
    p = native.from_workload(wl)
    g0 = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=100, amplitude=0.3)
    p.mf_set_state(0.05, torch.as_tensor(g0, device="cuda"), h=2e-5)
    default = p.mf_get_info()
    tu = p.mf_autotune(reps=5, force_iters=4)
    return {"workload": wl.name, "candidates": tu["candidates"],
            "default": {"rows_per_item": default["rows_per_item"], "grid": default["grid"],
                        "ms_per_rhs": tu["ms_per_rhs_default"]},
            "chosen": {"rows_per_item": tu["rows_per_item"], "two_field_rows": tu["zs_per_item"],
                       "grid": tu["grid"], "ms_per_rhs": tu["ms_per_rhs"]},
            "timing": "CUDA events, 5 launches of one right-hand side with 4 forced outside iterations"}


def _adaptive_decisions(log):
    """Accepted steps and per-step counts (k1, k2, k3) from a step log (k1 reused from the
    previous step's k4 when the log shows it was not evaluated)."""
    steps, counts, k4_prev = [], [], None
    for (t, h, _tn, outcome, iters, _err) in log:
        if outcome != 1:
            continue
        k1 = iters[0] if iters[0] >= 0 else k4_prev
        steps.append((t, h))
        counts += [int(k1), int(iters[1]), int(iters[2])]
        k4_prev = iters[3]
    return steps, counts


def adjoint_leg(native, W, torch, T: float = 0.04, ckpt: int = 20):
    """Secondary line: the gradient of the film-solve loss on the gradient workload (512^2 film
    in a 1024^2 grid, n = 30, lognormal jc map, 16 h_e knots on [0, T], a checkpoint every `ckpt`
    steps), FP32 transforms, against the same frozen forward alone and the plain FP64 forward and
    gradient.  The frozen decisions (accepted steps and per-call counts) are the oracle's adaptive
    run stored in tests/golden, else this GPU's own FP64 adaptive run.  Target: h_z(T) of this
    GPU's FP64 adaptive run with the second jc map (seed 6) (the frozen steps of one jc map are
    unstable for the other).  The calls are host-ordered launches, timed with the host clock
    around each call (each waits for its stream)."""
    import numpy as np
    wl = W.adjoint_film(1024, precision=1, T=T)
    path = os.path.join(ROOT, "tests", "golden", f"adjoint_{wl.name}.json")
    source = None
    if os.path.exists(path):
        ref = json.load(open(path))
        if abs(ref["T"] - T) < 1e-15:
            steps, iters = [tuple(x) for x in ref["steps"]], ref["counts"]
            source = "the oracle's adaptive run (tests/golden)"
    if source is None:
        pa = native.from_workload(wl, precision=0)
        pa.mf_advance(T)
        steps, iters = _adaptive_decisions(pa.mf_get_log())
        source = "this GPU's adaptive FP64 run"
        del pa
    g0 = torch.zeros((wl.ny, wl.nx), dtype=torch.float64, device="cuda")
    target = torch.zeros_like(g0)
    p6 = native.from_workload(wl, precision=0, jc_map=W.jc_map_lognormal((wl.ny, wl.nx), seed=6, sigma=0.2))
    p6.mf_advance(T)
    p6.mf_readout(native.MF_READ_HZ, out=target)
    del p6
    out = {"workload": wl.name, "steps": len(steps), "T": T, "ckpt_every": ckpt,
           "decisions": source, "mean_iterations_per_call": float(np.mean(iters))}
    for prec in (1, 0):
        wl.precision = prec
        p = native.from_workload(wl)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        L, _, _, _ = p.mf_film_solve_gradient(g0, target, steps, iters, ckpt, grad=False)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - w0
        w0 = time.perf_counter()
        L2, jcbar, kb, _ = p.mf_film_solve_gradient(g0, target, steps, iters, ckpt, grad=True)
        torch.cuda.synchronize()
        t_grad = time.perf_counter() - w0
        tag = "f32" if prec else "f64"
        out[tag] = {"loss": L, "forward_s": t_fwd, "gradient_s": t_grad,
                    "gradient_per_forward": t_grad / t_fwd, "knots_bar": kb,
                    "jcbar_l2": float(torch.linalg.norm(jcbar))}
    out["f32_gradient_vs_f64_forward"] = out["f64"]["forward_s"] / out["f32"]["gradient_s"]
    out["f32_gradient_vs_f64_gradient"] = out["f64"]["gradient_s"] / out["f32"]["gradient_s"]
    out["value"] = 1.0 / out["f32"]["gradient_s"]
    out["unit"] = "gradients/s"
    return out


def batch_leg(native, W, torch, count: int = 256, steps: int = 6, warmup: int = 2,
              max_side: int = 512):
    """Secondary line: a sweep of `count` independent films (seeded shapes, sides 64..512 cells,
    grids twice the film, n in {19, 30, 50}, ramp amplitudes in [0.2, 1]), FP32 transforms,
    advanced by one mf_advance_batch call (films smaller than the GPU in shared persistent
    launches, the others in launches of their own).  Beside it, a second copy of the same films
    in the same states advanced one after the other (one launch each): the two do the same
    work (a batched film's result is bit-identical to its own launch's).  Value = right-hand
    sides of all films per second."""
    wls = W.film_batch(count, seed=3, max_side=max_side, precision=1)
    sets = []
    for _ in range(2):
        ps = [native.from_workload(wl) for wl in wls]
        for p in ps:
            p.mf_set_state(0.0, None, h=1e-3)
        native.advance_batch(ps, [1.0] * count, max_attempts=warmup)
        sets.append(ps)
    torch.cuda.synchronize()

    def timed(ps, run):
        i0 = [p.mf_get_info() for p in ps]
        w0 = time.perf_counter()
        run()
        torch.cuda.synchronize()
        sec = time.perf_counter() - w0
        i1 = [p.mf_get_info() for p in ps]
        n_rhs = sum(b["n_rhs"] - a["n_rhs"] for a, b in zip(i0, i1))
        n_it = sum(b["n_iters"] - a["n_iters"] for a, b in zip(i0, i1))
        # (19 + 14 I) M per right-hand side, M = one FP32 field of the film's grid
        alg = sum(rhs_bytes(b["n_rhs"] - a["n_rhs"], b["n_iters"] - a["n_iters"], wl.nx * wl.ny * 4.0)
                  for a, b, wl in zip(i0, i1, wls))
        return n_rhs, n_it, sec, alg

    ps, qs = sets
    n_rhs, n_it, sec, alg = timed(ps, lambda: native.advance_batch(ps, [1.0] * count, max_attempts=steps))

    def one_by_one():
        for q in qs:
            q.mf_advance(1.0, max_attempts=steps)

    s_rhs, _, s_sec, _ = timed(qs, one_by_one)
    # the batched FP32 form against the plain FP64 solver on the same films (the first n64 of
    # the sweep, both advanced by one mf_advance_batch call from the same start)
    import dataclasses
    n64 = min(32, count)
    rates = {}
    for prec in (1, 0):
        sub = [dataclasses.replace(wl, precision=prec) for wl in wls[:n64]]
        rs = [native.from_workload(wl) for wl in sub]
        for r in rs:
            r.mf_set_state(0.0, None, h=1e-3)
        native.advance_batch(rs, [1.0] * n64, max_attempts=warmup)
        torch.cuda.synchronize()
        i0 = [r.mf_get_info() for r in rs]
        w0 = time.perf_counter()
        native.advance_batch(rs, [1.0] * n64, max_attempts=steps)
        torch.cuda.synchronize()
        el = time.perf_counter() - w0
        rates[prec] = sum(r.mf_get_info()["n_rhs"] - a["n_rhs"] for r, a in zip(rs, i0)) / el
        del rs
    cells = sum(wl.nx * wl.ny for wl in wls)
    name = f"film_batch_seed3_{count}" + ("" if max_side == 512 else f"_max{max_side}")
    return {"workload": name, "value": n_rhs / sec, "unit": UNIT,
            "films": count, "grid_cells": cells, "steps_per_film": steps,
            "mean_outside_iterations": n_it / max(n_rhs, 1),
            "algorithmic_bytes": alg, "achieved_gbs": alg / sec / 1e9,
            "one_launch_per_film": {"value": s_rhs / s_sec, "unit": UNIT, "same_work": s_rhs == n_rhs,
                                    "note": "a copy of the same films in the same states, advanced one after the other"},
            "speedup": (n_rhs / sec) / (s_rhs / s_sec),
            "fp64_subset": {"films": n64, "f32_rhs_per_s": rates[1], "f64_rhs_per_s": rates[0],
                            "speedup_of_f32_form": rates[1] / rates[0],
                            "note": "the first films of the sweep in both precisions, one mf_advance_batch "
                                    "call each (FP32 within 2e-4 of the oracle, FP64 within 1e-6)"},
            "timing": "host wall clock around one mf_advance_batch call"}


def full_ramp_leg(native, W, torch, precision: int):
    """Full ramp of the square film (64^2 cells in 128^2, n = 19, h_e 0 -> 0.5 over [0, 1]) on
    the GPU, timed end to end, with its error against the free-running FP64 oracle."""
    import numpy as np
    from oracle.bs23 import BS23
    from oracle.waveform import Waveform
    wl = W.square_film_128(precision=precision)
    p = native.from_workload(wl)
    t_out = np.linspace(0.1, 1.0, 10)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    m, hz = p.mf_run_ramp(t_out, want_fields=True)
    torch.cuda.synchronize()
    sec = time.perf_counter() - w0
    info = p.mf_get_info()
    o = _oracle_problem(wl)
    s = BS23(o.rhs, o.wf, rtol=wl.rtol, atol=wl.atol, on_accept=o.accept, on_attempt=o.begin_attempt)
    s.start(0.0, np.zeros((wl.ny, wl.nx)), 1.0)
    c0 = time.perf_counter()
    s.advance(1.0)
    cpu_sec = time.perf_counter() - c0
    hz_ref = o.hz(1.0, s.y)
    hz_gpu = hz[-1].cpu().numpy().reshape(wl.ny, wl.nx)
    return {"workload": wl.name, "transforms": "f32" if precision else "f64", "seconds": sec,
            "accepted_steps": info["n_accepted"], "rejected_steps": info["n_rejected"],
            "rhs_evals": info["n_rhs"],
            "rel_err_hz": float(np.linalg.norm(hz_gpu - hz_ref) / np.linalg.norm(hz_ref)),
            "rel_err_m": float(abs(m[-1, 0] - o.magnetization(s.y)) / abs(o.magnetization(s.y))),
            "oracle_seconds": cpu_sec}


def golden_ramp_leg(native, W, torch, which: str):
    """Full ramp of a stated workload on the GPU (FP32 transforms, FP64 state), free running from
    a zero state, timed end to end (mf_run_ramp with its readouts), with its relative L2 errors
    against the FP64 oracle's stored ramp (tests/golden/, written by make_ramp_goldens.py)."""
    import numpy as np
    wl = W.rect_film_2048(precision=1) if which == "film" else W.cube_bulk(128, precision=1)
    path = os.path.join(ROOT, "tests", "golden", f"ramp_{wl.name}.npz")
    if not os.path.exists(path):
        return {"workload": wl.name, "skipped": "no stored oracle ramp"}
    ref = np.load(path)
    meta = json.load(open(path.replace(".npz", ".json")))
    p = native.from_workload(wl)
    t_out = ref["t_out"]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    m, fields = p.mf_run_ramp(t_out, want_fields=True)
    torch.cuda.synchronize()
    sec = time.perf_counter() - w0
    info = p.mf_get_info()
    stride = meta["field_stride"]
    errs, num, den = [], 0.0, 0.0
    for tf, fref in zip(ref["t_fields"], ref["fields"]):
        k = int(np.argmin(np.abs(t_out - tf)))
        f = fields[k].cpu().numpy()
        if wl.dim == 2:
            f = f.reshape(wl.ny, wl.nx)[::stride, ::stride]
        else:
            lo, hi = wl.nx // 4 - 4, 3 * wl.nx // 4 + 4
            f = f.reshape(3, wl.nz, wl.ny, wl.nx)[:, lo:hi:stride, lo:hi:stride, lo:hi:stride]
        d2, n2 = float(((f - fref) ** 2).sum()), float((fref ** 2).sum())
        errs.append((d2 / n2) ** 0.5)
        num, den = num + d2, den + n2
    mref = ref["m"].reshape(len(t_out), -1)
    m_err = float(np.linalg.norm(m - mref) / np.linalg.norm(mref))
    return {"workload": wl.name, "transforms": "f32", "t_end": float(t_out[-1]), "seconds": sec,
            "accepted_steps": info["n_accepted"], "rejected_steps": info["n_rejected"],
            "rhs_evals": info["n_rhs"], "outside_iterations": info["n_iters"],
            "rel_err_m_loop": m_err, "rel_err_field_spacetime": (num / den) ** 0.5,
            "rel_err_field_per_snapshot": errs, "field": meta["field"],
            "tolerance": {"m_loop": 2e-4, "field_spacetime": 4e-4 if wl.dim == 2 else 2e-4},
            "oracle_seconds": meta["oracle_seconds"], "oracle_fft_workers": meta["fft_workers"],
            "oracle_steps": meta["attempts"]}


def fp64_leg(native, W, torch, steps: int = 5, warmup: int = 3):
    """Secondary line: the same film and start with FP64 transforms (the plain FP64 solver),
    timed like the main line, and the precision form's speed-up over it."""
    wl = W.rect_film_2048(precision=0)
    p = native.from_workload(wl)
    g0 = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=100, amplitude=0.3)
    p.mf_set_state(T_START, torch.as_tensor(g0, device="cuda"), h=H_START)
    p.mf_advance(1.0, max_attempts=warmup)
    torch.cuda.synchronize()
    i0 = p.mf_get_info()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(p.stream)
    p.mf_advance(1.0, max_attempts=steps)
    e1.record(p.stream)
    torch.cuda.synchronize()
    i1 = p.mf_get_info()
    sec = e0.elapsed_time(e1) / 1000.0
    n_rhs, n_it = i1["n_rhs"] - i0["n_rhs"], i1["n_iters"] - i0["n_iters"]
    M = wl.nx * wl.ny * 8.0
    alg = rhs_bytes(n_rhs, n_it, M)
    peak, kind = hbm_peak()
    return {"workload": wl.name, "transforms": "f64", "value": n_rhs / sec, "unit": UNIT,
            "steps": i1["n_attempts"] - i0["n_attempts"], "rhs_evals": n_rhs,
            "mean_outside_iterations": n_it / max(n_rhs, 1),
            "ms_per_round_trip": 1000.0 * sec / (2 * n_rhs + 2 * n_it),
            "roofline": {"bound": "hbm", "achieved": alg / sec / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / sec / 1e9 / peak, "peak_kind": kind,
                         "bytes_model": "(19 + 14 I) M per RHS, M = 2048^2 x 8 B"}}


def cufft_leg(torch, n: int = 2048, reps: int = 50):
    """Reference point only (the library never calls it): cuFFT round trips
    irfft2(M * rfft2(x)) of an n x n real field through torch.fft, in FP32 and FP64, CUDA-event
    timed after warm-up."""
    out = {"grid": [n, n], "note": "torch.fft (cuFFT) round trip with a pointwise multiplier; "
                                   "timed beside the library as a reference point only"}
    for dt, name in ((torch.float32, "f32"), (torch.float64, "f64")):
        x = torch.randn(n, n, device="cuda", dtype=dt)
        mult = torch.rand(n, n // 2 + 1, device="cuda", dtype=dt)

        def rt():
            return torch.fft.irfft2(torch.fft.rfft2(x) * mult, s=(n, n))
        for _ in range(5):
            rt()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            rt()
        e1.record()
        torch.cuda.synchronize()
        out[f"ms_per_round_trip_{name}"] = e0.elapsed_time(e1) / reps
    return out


def cufft3_leg(torch, n: int, reps: int = 10):
    """Reference point only (the library never calls it): the transform floor of one vector
    round trip of the bulk solver through torch.fft (cuFFT), irfftn(M * rfftn(h)) of the three
    components of an n^3 FP32 field with one real multiplier (a lower bound on the pointwise work
    of a spectral curl), CUDA-event timed after warm-up."""
    x = torch.randn(3, n, n, n, device="cuda", dtype=torch.float32)
    mult = torch.rand(n, n, n // 2 + 1, device="cuda", dtype=torch.float32)

    def rt():
        return torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)) * mult, s=(n, n, n), dim=(1, 2, 3))
    for _ in range(3):
        rt()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        rt()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del x, mult
    torch.cuda.empty_cache()
    return {"grid": [n, n, n], "ms_per_vector_round_trip_f32": ms,
            "note": "torch.fft (cuFFT) forward and inverse of 3 components with one pointwise "
                    "multiplier; timed beside the library as a reference point only"}


def combine_ranks(dist, sec: float, n_rhs: int, e2e_rate: float, device):
    """Whole-job figures of a multi-rank run: the slowest rank's timed seconds, the evaluations of
    all ranks and the sum of the ranks' end-to-end rates (the replicas run side by side).
    `dist` is torch.distributed with an initialised process group, or None for one rank."""
    if dist is None:
        return sec, float(n_rhs), e2e_rate
    import torch
    mx = torch.tensor([sec], device=device, dtype=torch.float64)
    sm = torch.tensor([float(n_rhs), e2e_rate], device=device, dtype=torch.float64)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[0]), float(sm[1])


def cores_used() -> int:
    """Host threads of the oracle's transforms (scipy.fft workers); its elementwise steps run on
    one thread."""
    from oracle import _fft
    return _fft.workers()


T_START = 0.05          # the timed steps start mid-cycle from a seeded critical-state film
H_START = 2e-5


def bench_config(wl) -> dict:
    """The workload both arms time (identical in the two JSON lines)."""
    return {"workload": wl.name, "grid": [wl.nx, wl.ny], "film_cells": [wl.nx // 2, wl.ny // 4],
            "n": wl.n, "he": "0.8 sin(2 pi t)", "rtol": wl.rtol, "atol": wl.atol,
            "iter_tol": wl.iter_tol, "outside_iteration": "converged, warm-started (Section 2.2)",
            "start": f"seeded critical-state film at t = {T_START}, h = {H_START}, after the warm-up",
            "l2": "working set > L2 (no flush)"}


class _Enough(Exception):
    pass


def oracle_rhs_sample(warmup: int, count: int = 0, budget_s: float = 0.0):
    """The FP64 oracle on the benchmark workload and start state: its own Bogacki-Shampine
    integrator and warm-started outside iteration from t = T_START, `warmup` right-hand sides
    untimed, then `count` timed right-hand sides (or as many as `budget_s` seconds allow, at least
    two).  Returns (RHS per second, timed RHS, seconds, mean outside iterations, t reached)."""
    import numpy as np
    import workloads as W
    from oracle.bs23 import BS23
    wl = W.rect_film_2048(precision=0)
    o = _oracle_problem(wl)
    g0 = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=100, amplitude=0.3)
    marks = {}
    iters = []

    def rhs(t, y, seg, force):
        if len(iters) == warmup:
            marks["t0"] = time.perf_counter()
        r = o.rhs(t, y, seg, force)
        iters.append(r[1])
        n = len(iters) - warmup
        if n > 0:
            marks["t1"] = time.perf_counter()
            if (count and n >= count) or (budget_s and n >= 2 and marks["t1"] - marks["t0"] > budget_s):
                raise _Enough
        return r

    s = BS23(rhs, o.wf, rtol=wl.rtol, atol=wl.atol, h0=H_START, on_accept=o.accept,
             on_attempt=o.begin_attempt)
    s.start(T_START, g0, 1.0)
    try:
        s.advance(1.0)
    except _Enough:
        pass
    n = len(iters) - warmup
    el = marks["t1"] - marks["t0"]
    return n / el, n, el, float(np.mean(iters[warmup:])), s.t


def run_reference(args):
    """The oracle (FP64, CPU) on the same workload and start state as the GPU arm, W right-hand
    sides of warm-up, then exactly K timed right-hand sides (one step of this arm = one
    right-hand side, the unit of the metric)."""
    import workloads as W
    wl = W.rect_film_2048(precision=0)
    W_, K = max(1, args.warmup), max(1, args.steps)
    rate, n, el, mean_it, t_reached = oracle_rhs_sample(W_, count=K)
    cores = cores_used()
    sample = (f"{K} right-hand sides (after {W_} of warm-up) of the oracle's own BS23 run of the "
              f"{wl.nx}x{wl.ny} film from the GPU arm's start state: converged warm-started outside "
              f"iterations, mean {mean_it:.1f}; transforms on {cores} threads, elementwise steps on one")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W_, "ms_per_step": 1000.0 * el / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(wl),
            "run": {"step": "one right-hand side", "mean_outside_iterations": mean_it,
                    "t_reached": t_reached},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the bulk and full-ramp legs")
    ap.add_argument("--grid", type=int, default=2048, help="film grid (2048 is the benchmark)")
    ap.add_argument("--no-tune", action="store_true",
                    help="--only bulk: keep the size rules' item shape (no mf_autotune launches)")
    ap.add_argument("--only", choices=["batch", "adjoint", "ramps", "fp64", "cufft", "bulk"],
                    help="run one secondary leg alone")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-max-side", type=int, default=512)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import numpy as np
    import torch

    import workloads as W
    from paper_1801_04869_gb300 import native

    torch.cuda.set_device(local)
    if args.only == "batch":
        if rank == 0:
            print(json.dumps(batch_leg(native, W, torch, count=args.batch_count,
                                       max_side=args.batch_max_side)))
        return
    if args.only == "adjoint":
        if rank == 0:
            print(json.dumps(adjoint_leg(native, W, torch)))
        return
    if args.only == "ramps":
        if rank == 0:
            print(json.dumps([golden_ramp_leg(native, W, torch, w) for w in ("film", "cube")]))
        return
    if args.only == "fp64":
        if rank == 0:
            print(json.dumps(fp64_leg(native, W, torch)))
        return
    if args.only == "cufft":
        if rank == 0:
            print(json.dumps(cufft_leg(torch)))
        return
    if args.only == "bulk":
        # the cube leg alone: --grid 128 or 256 (the cube has half the grid's cells per side)
        if rank == 0:
            print(json.dumps(bulk_leg(native, W, torch, steps=args.steps, warmup=args.warmup,
                                      n_grid=args.grid if args.grid <= 512 else 128,
                                      tune=not args.no_tune)))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    wl = W.rect_film_2048(precision=1, n_grid=args.grid)
    p = native.from_workload(wl)
    stream = p.stream
    ncell = wl.nx * wl.ny
    M = ncell * 4.0                                     # one FP32 real field

    # start mid-cycle from a seeded critical-state film so that the warm-up absorbs the cold
    # start of the outside iteration
    g0 = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=100 + rank, amplitude=0.3)
    y = torch.as_tensor(g0, device="cuda")
    p.mf_set_state(T_START, y, h=H_START)
    p.mf_advance(1.0, max_attempts=max(1, args.warmup))
    torch.cuda.synchronize()

    def counters():
        i = p.mf_get_info()
        return i["n_rhs"], i["n_iters"], i["n_attempts"]

    r0, it0, a0 = counters()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as ck:
        ev0.record(stream)
        p.mf_advance(1.0, max_attempts=args.steps)     # one persistent launch, K step attempts
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    r1, it1, a1 = counters()
    n_rhs, n_it, n_att = r1 - r0, it1 - it0, a1 - a0
    # the integrator may stop early only at t = 1 (end of the cycle)
    t_now, _ = p.mf_get_state()

    # end-to-end through the public API with the solver state resident in pinned host memory:
    # every step restores the checkpoint (state, first-same-as-last derivative, warm start, step
    # size, counters) from the host, advances one step, saves it back and reads m_z, so the
    # steps follow the timed region's trajectory and do the same work
    nblob = native.load().mf_checkpoint_bytes(p.h)
    blob = torch.empty(nblob, dtype=torch.uint8).pin_memory()
    p.mf_checkpoint_save(blob)
    e2e_steps = max(3, args.steps // 2)
    re0, ie0, _ = counters()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        p.mf_checkpoint_restore(blob)
        p.mf_advance(1.0, max_attempts=1)
        p.mf_checkpoint_save(blob)
        m = p.mf_readout(native.MF_READ_MOMENT)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - w0
    re1, ie1, _ = counters()
    e2e_rate = (re1 - re0) / e2e_s

    sec = ms / 1000.0
    sec_all, rhs_all, e2e_all = combine_ranks(dist, sec, n_rhs, e2e_rate, "cuda")

    if rank == 0:
        peak, peak_kind = hbm_peak()
        mean_it = n_it / max(n_rhs, 1)
        alg = rhs_bytes(n_rhs, n_it, M)
        achieved = alg / sec / 1e9
        traffic_ratio = profiled_traffic("film_kernel_f32", wl.name)
        cpu = None
        if not args.no_cpu:
            rate, n, el, mit, _ = oracle_rhs_sample(2, budget_s=15.0)
            cpu = {"value": rate, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
                   "sample": f"{n} right-hand sides (after 2 of warm-up) of the FP64 oracle's own "
                             f"BS23 run of the {wl.nx}x{wl.ny} film from this line's start state, "
                             f"converged outside iterations (mean {mit:.1f}); {el:.1f} s; transforms "
                             f"on {cores_used()} threads, elementwise steps on one"}
        info = p.mf_get_info()
        bulk = bulk_leg(native, W, torch) if not args.no_extra else None
        bulk_256 = bulk_leg(native, W, torch, n_grid=256) if not args.no_extra else None
        tune = autotune_leg(native, W, torch, args.grid) if not args.no_extra else None
        adj = adjoint_leg(native, W, torch) if not args.no_extra else None
        batch = batch_leg(native, W, torch) if not args.no_extra else None
        ramps = None
        if not args.no_extra:
            ramps = [full_ramp_leg(native, W, torch, prec) for prec in (0, 1)]
            ramps += [golden_ramp_leg(native, W, torch, w) for w in ("film", "cube")]
        f64 = fp64_leg(native, W, torch) if not args.no_extra else None
        if f64 is not None:
            f64["speedup_of_f32_form"] = (n_rhs / sec) / f64["value"]
        cufft = cufft_leg(torch) if not args.no_extra else None
        if cufft is not None:
            cufft["library_ms_per_round_trip_f32"] = 1000.0 * sec / (2 * n_rhs + 2 * n_it)
            if f64 is not None:
                cufft["library_ms_per_round_trip_f64"] = f64["ms_per_round_trip"]
        line = {
            "metric": METRIC, "value": rhs_all / sec_all, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sec_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": bench_config(wl),
            "run": {"step": "one BS23 step attempt (3-4 right-hand sides, error norm, control)",
                    "state": "f64", "transforms": "f32",
                    "parallelism": "replicas" if world > 1 else "single", "t_end": t_now,
                    "step_attempts": n_att, "rhs_evals": n_rhs, "mean_outside_iterations": mean_it,
                    "grid_ctas": info["grid"], "threads": info["threads"],
                    "ms_per_round_trip": 1000.0 * sec / (2 * n_rhs + 2 * n_it)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": None if traffic_ratio is None else traffic_ratio * alg,
                         "traffic_note": "ncu dram bytes of a 1-step launch, scaled to this launch by its algorithmic bytes",
                         "kernel": "film_kernel<float> (persistent)",
                         "bytes_model": "(19 + 14 I) M per RHS, M = 2048^2 x 4 B"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_all, "unit": UNIT, "h2d_bytes_per_step": nblob,
                    "d2h_bytes_per_step": nblob + 8, "ms_per_step": 1000.0 * e2e_s / e2e_steps,
                    "note": "solver state in pinned host memory: each step restores the whole "
                            "checkpoint (state, derivative buffers, warm start, step log) from "
                            "the host, advances one step and saves it back, then reads m_z"},
            "gpu_launches": 1,
            "clocks": ck.summary(),
            "bulk": bulk,
            "bulk_256": bulk_256,
            "autotune": tune,
            "adjoint": adj,
            "batch": batch,
            "full_ramp": ramps,
            "fp64": f64,
            "cufft": cufft,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
