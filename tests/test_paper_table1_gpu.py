"""The paper's thin-disk example (Section 2.3, Table 1) on the GPU path.

A disk of radius 1 in D = [-2, 2]^2, power law n = 1000, rho_out = 1, h_e = t, integrated by the
library's BS23 (rtol 1e-3, atol 1e-6, outside-iteration tolerance 2e-4, lambda = 0.7) up to
h_e = 0.5.  The sheet current is compared in the L1 norm with the Bean critical state of a thin
disk (front radius b = 1 / cosh(2 h_e) in these units, |j| = 1 outside it and
(2/pi) arctan(r sqrt(1 - b^2) / sqrt(b^2 - r^2)) inside).  Table 1 of the paper reports
delta_j = 2.2 % on the 128^2 grid, 1.0 % on 256^2 and 0.9 % on 512^2
(tests/golden/table1_thin_disk.json).
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle.film2d import FilmProblem
from oracle.waveform import Waveform

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_thin_disk.json")))
HE = 0.5


def _disk_delta_j(n_grid: int, precision: int) -> float:
    L = 2.0
    mask = W.film_mask(n_grid, n_grid, L, L, "disk", radius=1.0)
    wl = W.Workload(f"disk_{n_grid}", 2, n_grid, n_grid, 1, L, L, 0.0, mask, n=1000.0, rho_out=1.0,
                    precision=precision, t0=0.0, t1=HE, he_knots=((0.0, 1.0), (0.0, 1.0)),
                    iter_max=3000, rtol=1e-3, atol=1e-6)
    p = native.from_workload(wl)
    p.mf_set_state(0.0, None, h=1e-3)
    p.mf_advance(HE)
    g = torch.zeros(n_grid * n_grid, dtype=torch.float64, device="cuda")
    t, _ = p.mf_get_state(g)
    assert t == pytest.approx(HE, abs=1e-12)
    g = g.cpu().numpy().reshape(n_grid, n_grid)
    # sheet current j = (d_y g, -d_x g) by the same smoothed spectral derivative (host, FP64)
    fp = FilmProblem(n_grid, n_grid, L, L, mask, n=1000.0, rho_out=1.0,
                     waveform=Waveform((0.0, 1.0), (0.0, 1.0)))
    jx, jy = fp.sheet_current(g)
    j = np.sqrt(jx ** 2 + jy ** 2)
    x = W.cell_centres(n_grid, L)
    r = np.sqrt(x[None, :] ** 2 + x[:, None] ** 2)
    inside = mask == 1
    b = 1.0 / math.cosh(2.0 * HE)
    rr = r[inside]
    jb = np.ones(rr.size)
    m = rr < b
    jb[m] = (2.0 / math.pi) * np.arctan(rr[m] * math.sqrt(1.0 - b * b) / np.sqrt(b * b - rr[m] ** 2))
    return 100.0 * np.abs(j[inside] - jb).sum() / jb.sum()


def _paper(grid: int) -> float:
    return next(r["delta_j_percent"] for r in GOLDEN["rows"] if r["grid"] == grid)


def test_thin_disk_128_fp64_matches_table1():
    dj = _disk_delta_j(128, precision=0)
    assert abs(dj - _paper(128)) < 0.4, dj


def test_thin_disk_256_fp32_matches_table1():
    dj = _disk_delta_j(256, precision=1)
    assert abs(dj - _paper(256)) < 0.3, dj


@pytest.mark.slow
def test_thin_disk_512_fp32_matches_table1():
    dj = _disk_delta_j(512, precision=1)
    assert abs(dj - _paper(512)) < 0.3, dj
