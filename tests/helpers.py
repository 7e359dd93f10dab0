"""Shared test helpers: build the same problem for the CUDA library and for the oracle."""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle.bulk3d import BulkProblem
from oracle.film2d import FilmProblem
from oracle.waveform import Waveform


def waveform_of(wl: W.Workload) -> Waveform:
    if wl.he_knots is not None:
        return Waveform(*wl.he_knots)
    return Waveform(sin_amp=wl.he_sin[0], sin_period=wl.he_sin[1])


def oracle_of(wl: W.Workload, **over):
    kw = dict(n=wl.n, rho_out=wl.rho_out, waveform=waveform_of(wl), jc=wl.jc if wl.jc_map is None
              else wl.jc_map, sigma=wl.sigma, iter_tol=wl.iter_tol, iter_max=wl.iter_max,
              gamma=wl.gamma)
    if wl.dim == 3 and wl.b0 > 0:
        kw["b0"] = wl.b0
    if wl.dim == 2:
        kw["lam"] = wl.lam
        kw.update(over)
        return FilmProblem(wl.nx, wl.ny, wl.Lx, wl.Ly, wl.mask, **kw)
    kw["he_dir"] = wl.vector_he
    kw.update(over)
    return BulkProblem(wl.nx, wl.ny, wl.nz, wl.Lx, wl.Ly, wl.Lz, wl.mask, **kw)


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def film_workload(nx, ny, L=(2.0, 2.0), shape="rect", precision=0, **kw) -> W.Workload:
    Lx, Ly = L
    dims = {k: kw.pop(k) for k in ("ax", "ay", "radius", "hole") if k in kw}
    m = W.film_mask(nx, ny, Lx, Ly, shape, **dims)
    base = dict(n=19.0, rho_out=1.0, precision=precision, t0=0.0, t1=1.0,
                he_knots=((0.0, 1.0), (0.0, 0.5)))
    base.update(kw)
    return W.Workload(f"film_{nx}x{ny}", 2, nx, ny, 1, Lx, Ly, 0.0, m, **base)
