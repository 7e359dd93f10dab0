"""The film-solve gradient at the size of the gradient workload: a 512^2 film in a 1024^2 grid,
n = 30, a lognormal jc map (seed 5), 16 h_e knots on [0, T], frozen decisions (accepted steps and
outside-iteration counts) of the oracle's own adaptive run, checkpoints every 20 steps, target
h_z(T) of an adaptive run with a second jc map (seed 6).  The target is rebuilt here by the
library's own FP64 adaptive run and checked against the stored target (counts, norm, sum and
64 sampled cells) before it is used.

* Against the stored FP64 oracle gradient (tests/golden/make_adjoint_golden.py): the loss, dL/d(knot
  values), dL/djc at 32 seeded cells of the film, and the directional derivatives along two seeded
  directions d = jc z.  FP64 transforms to 1e-8; FP32 transforms to the tolerance derived below.
* Against central differences of the GPU's own FP64 map for 8 of the 32 cells, every knot and
  both directions.  The map is deterministic (fixed reduction order), so rounding limits the
  differences only at the 1e-9 level; its curvature does at larger steps: with n = 30 near the
  critical state and 794 explicit steps, a knot step of 1e-4 moves the central difference of
  the fourth knot's derivative by 7 % and 1e-5 by 0.06 %, while 1e-6 and 1e-7 agree with the
  gradient to 6e-6 and 3e-7.  Steps: 1e-6 relative for jc, 1e-7 for the knot values and the
  directions; gates 1e-4 (cells) and 1e-5 (knots, directions), relative (the deviations are
  printed).

FP32 tolerance: every right-hand side of the FP32 form is within 2e-4 of FP64 (relative L2), and
the gradient of a solve of ~800 steps sums ~2400 vector-Jacobian products and as many forward
evaluations whose rounding errors do not cancel in a loss that is itself a small difference
(h_z(T) - target): the measured deviation is recorded in the test output and the bound is 2e-2.
"""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
FD_CELLS = 8
EPS_JC = 1e-6          # relative step of a cell's jc
EPS = 1e-7             # step of a knot value; step along a direction d = jc z


def _stored():
    wl0 = W.adjoint_film(1024, precision=0, T=0.04)
    path = os.path.join(HERE, "golden", f"adjoint_{wl0.name}.json")
    if not os.path.exists(path):
        pytest.skip("no stored oracle gradient")
    return json.load(open(path))


def _setup(ref, precision):
    wl = W.adjoint_film(ref["grid"][0], precision=precision, T=ref["T"])
    steps = [tuple(s) for s in ref["steps"]]
    counts = ref["counts"]
    g0 = torch.zeros((wl.ny, wl.nx), dtype=torch.float64, device="cuda")
    target = _target(ref)
    p = native.from_workload(wl)
    return wl, p, g0, target, steps, counts


def _target(ref):
    """h_z(T) of the FP64 adaptive run with the second jc map, checked against the stored one."""
    wl6 = W.adjoint_film(ref["grid"][0], precision=0, T=ref["T"])
    jc6 = W.jc_map_lognormal((wl6.ny, wl6.nx), seed=ref["target_jc_seed"], sigma=0.2)
    p6 = native.from_workload(wl6, jc_map=jc6)
    p6.mf_advance(ref["T"])
    info = p6.mf_get_info()
    target = torch.zeros((wl6.ny, wl6.nx), dtype=torch.float64, device="cuda")
    p6.mf_readout(native.MF_READ_HZ, out=target)
    t = target.cpu().numpy()
    assert (info["n_attempts"], info["n_accepted"]) == (ref["target_attempts"], ref["target_accepted"])
    vals = np.array([t[iy, ix] for iy, ix in ref["cells"] + ref["out_cells"]])
    want = np.array(ref["target_cells"] + ref["target_out_cells"])
    assert np.max(np.abs(vals - want)) <= 1e-9 * np.abs(want).max()
    assert abs(np.linalg.norm(t) - ref["target_l2"]) <= 1e-9 * ref["target_l2"]
    return target


def _compare(ref, wl, L, cb, vb):
    """Relative deviations from the stored gradient.  A directional derivative <dL/djc, d> over
    all cells with random signs cancels to a small fraction of |dL/djc| |d|, so its deviation is
    measured against that bound (Cauchy-Schwarz), not against its own small value."""
    cells = [tuple(c) for c in ref["cells"]]
    cbv = np.array([cb[iy, ix] for iy, ix in cells])
    dirs = [wl.jc_map * W.rng(s).standard_normal(wl.jc_map.shape) for s in ref["direction_seeds"]]
    dd = np.array([float((cb * d).sum()) for d in dirs])
    scale = np.array([ref["jcbar_l2"] * float(np.linalg.norm(d)) for d in dirs])
    return {"loss": abs(L - ref["loss"]) / abs(ref["loss"]),
            "knots": float(np.linalg.norm(np.array(vb) - ref["knots_bar"]) / np.linalg.norm(ref["knots_bar"])),
            "cells": float(np.linalg.norm(cbv - ref["jcbar_cells"]) / np.linalg.norm(ref["jcbar_cells"])),
            "directional": float(np.max(np.abs(dd - ref["directional"]) / scale)),
            "l2": abs(float(np.linalg.norm(cb)) - ref["jcbar_l2"]) / ref["jcbar_l2"]}


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 2e-2)])
def test_gradient_matches_the_stored_oracle_gradient(precision, tol):
    ref = _stored()
    wl, p, g0, target, steps, counts = _setup(ref, precision)
    L, cb, vb, _ = p.mf_film_solve_gradient(g0, target, steps, counts, ref["ckpt_every"])
    err = _compare(ref, wl, L, cb.cpu().numpy(), vb)
    print(f"precision {precision}: {len(steps)} steps, relative deviations {err}")
    for k, v in err.items():
        assert v < tol, (k, v)


def test_gradient_matches_central_differences_of_the_gpu_map():
    ref = _stored()
    wl, p, g0, target, steps, counts = _setup(ref, 0)
    C = ref["ckpt_every"]
    L0, cb, vb, _ = p.mf_film_solve_gradient(g0, target, steps, counts, C)
    cb = cb.cpu().numpy()
    jc = torch.as_tensor(wl.jc_map, device="cuda")
    kv = list(wl.he_knots[1])

    def loss(jc_map=None, knots=None):
        p.mf_set_jc_map(jc if jc_map is None else jc_map)
        p.mf_set_knot_values(kv if knots is None else knots)
        return p.mf_film_solve_gradient(g0, target, steps, counts, C, grad=False)[0]

    assert loss() == L0                                        # the map is deterministic
    worst = worst_k = 0.0
    for iy, ix in [tuple(c) for c in ref["cells"][:FD_CELLS]]:
        dj = EPS_JC * float(wl.jc_map[iy, ix])
        e = torch.zeros_like(jc)
        e[iy, ix] = dj
        fd = (loss(jc + e) - loss(jc - e)) / (2 * dj)
        if fd != 0.0:                                   # a cell the loss does not feel
            worst = max(worst, abs(fd - cb[iy, ix]) / abs(fd))
        assert abs(fd - cb[iy, ix]) <= 1e-4 * abs(fd) + 1e-6 * np.abs(cb).max(), (iy, ix, fd, cb[iy, ix])
    def knot_fd(k, eps):
        up, dn = list(kv), list(kv)
        up[k] += eps
        dn[k] -= eps
        return (loss(knots=up) - loss(knots=dn)) / (2 * eps)

    for k in range(len(kv)):
        fd = knot_fd(k, EPS)
        worst_k = max(worst_k, abs(fd - vb[k]) / abs(fd))
        assert abs(fd - vb[k]) <= 1e-5 * abs(fd) + 1e-8 * np.abs(vb).max(), (k, fd, vb[k])
    worst_d = 0.0
    for s in ref["direction_seeds"]:
        d = torch.as_tensor(wl.jc_map * W.rng(s).standard_normal(wl.jc_map.shape), device="cuda")
        fd = (loss(jc + EPS * d) - loss(jc - EPS * d)) / (2 * EPS)
        an = float((cb * d.cpu().numpy()).sum())
        worst_d = max(worst_d, abs(fd - an) / abs(fd))
        assert abs(fd - an) <= 1e-5 * abs(fd), (s, fd, an)
    print(f"central differences: worst relative deviation cells {worst:.2e}, knots {worst_k:.2e}, "
          f"directions {worst_d:.2e}")


def test_frozen_map_is_the_adaptive_solve():
    """The differentiated map is the solver's own trajectory: the FP64 adaptive run of the
    workload takes the stored decisions (the same attempts and accepted steps), and the frozen
    forward with those steps and counts reaches its h_z(T).  They differ only where a step ends
    on an h_e knot (15 of the 794): there the integrator evaluates a k4 that the next step
    discards (h_e_dot jumps) and warm-starts the recomputed k1 from it, while the frozen map,
    which has no k4 call, warm-starts k1 from k3; with the same iteration counts the two starts
    leave differences at the level of the stop tolerance (measured 7.6e-6 relative L2)."""
    ref = _stored()
    wl = W.adjoint_film(ref["grid"][0], precision=0, T=ref["T"])
    pa = native.from_workload(wl)
    pa.mf_advance(ref["T"])
    info = pa.mf_get_info()
    assert (info["n_attempts"], info["n_accepted"]) == (ref["adaptive_attempts"], ref["n_steps"])
    hz_a = torch.zeros((wl.ny, wl.nx), dtype=torch.float64, device="cuda")
    pa.mf_readout(native.MF_READ_HZ, out=hz_a)
    del pa
    p = native.from_workload(wl)
    g0 = torch.zeros_like(hz_a)
    hz_f = torch.zeros_like(hz_a)
    p.mf_film_solve_gradient(g0, g0, [tuple(s) for s in ref["steps"]], ref["counts"], ref["ckpt_every"],
                             grad=False, hz_out=hz_f)
    err = float(torch.linalg.norm(hz_f - hz_a) / torch.linalg.norm(hz_a))
    print(f"frozen forward against the adaptive run: h_z(T) relative L2 {err:.2e}")
    assert err < 3e-5, err
