"""Seeded synthetic inputs for the thin-film (2D) and bulk (3D) magnetization problems.

This module builds inputs only: cell-centred domain masks, plausible states (stream function
g or field h), per-cell critical-current maps and the parameter sets of the standard workloads.
It holds none of the method's arithmetic (no transform, no power law, no iteration, no
integrator), so both the CUDA path and the CPU oracle can draw their inputs from it.

Grids are cell-centred on the periodic box D = [-Lx,Lx] x [-Ly,Ly] (x [-Lz,Lz]):
x_i = -Lx + (i + 1/2) dx with dx = 2 Lx / nx.  Arrays are indexed [y, x] in 2D and
[z, y, x] in 3D (x fastest), matching the row-major device layout.

Mask classes (Section 2.2 and Section 3.1 of the paper):
  0  free space inside D (Ohm law with rho_out, the outside iteration acts here)
  1  superconductor (power law)
  2  normal conductor with Ohm law that is not iterated (filled hole in 2D, cutting layer in 3D)
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASK_OUT, MASK_SC, MASK_NORMAL = 0, 1, 2


# --------------------------------------------------------------------------------------------
# counter-based seeding (splitmix64) so that any consumer reproduces the same shapes
# --------------------------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(state: int) -> tuple[int, int]:
    """One step of splitmix64 (Steele, Lea and Flood 2014): returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def rng(seed: int) -> np.random.Generator:
    """numpy generator whose seed is mixed through splitmix64."""
    _, s = splitmix64(seed & _M64)
    return np.random.default_rng(s)


# --------------------------------------------------------------------------------------------
# grids and masks
# --------------------------------------------------------------------------------------------
def cell_centres(n: int, L: float) -> np.ndarray:
    d = 2.0 * L / n
    return -L + (np.arange(n) + 0.5) * d


def film_mask(nx: int, ny: int, Lx: float, Ly: float, shape: str = "rect", *,
              ax: float = 1.0, ay: float = 1.0, radius: float = 1.0,
              cx: float = 0.0, cy: float = 0.0,
              hole: tuple[float, float, float] | None = None) -> np.ndarray:
    """uint8 (ny, nx) mask of a film: 'rect' |x-cx|<=ax, |y-cy|<=ay, or 'disk' of `radius`.

    `hole=(hx, hy, hr)` marks a circular hole as class 2 (filled, Ohm law, not iterated).
    Cells are classified by their centres.
    """
    x = cell_centres(nx, Lx)[None, :]
    y = cell_centres(ny, Ly)[:, None]
    if shape in ("rect", "square"):
        inside = (np.abs(x - cx) <= ax) & (np.abs(y - cy) <= ay)
    elif shape == "disk":
        inside = (x - cx) ** 2 + (y - cy) ** 2 <= radius ** 2
    else:
        raise ValueError(f"unknown film shape {shape!r}")
    m = np.where(inside, MASK_SC, MASK_OUT).astype(np.uint8)
    if hole is not None:
        hx, hy, hr = hole
        m[(x - hx) ** 2 + (y - hy) ** 2 <= hr ** 2] = MASK_NORMAL
    return m


def bulk_mask(nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float, shape: str = "box", *,
              ax: float = 0.5, ay: float = 0.5, az: float = 0.5,
              r_in: float = 0.0, r_out: float = 1.0) -> np.ndarray:
    """uint8 (nz, ny, nx) mask: 'box' |x|<=ax,|y|<=ay,|z|<=az; 'ball' r_in <= |r| <= r_out;
    'slab' |x| <= ax (spanning the periodic box in y and z)."""
    x = cell_centres(nx, Lx)[None, None, :]
    y = cell_centres(ny, Ly)[None, :, None]
    z = cell_centres(nz, Lz)[:, None, None]
    if shape == "box":
        inside = (np.abs(x) <= ax) & (np.abs(y) <= ay) & (np.abs(z) <= az)
    elif shape == "ball":
        r2 = x * x + y * y + z * z
        inside = (r2 <= r_out ** 2) & (r2 >= r_in ** 2)
    elif shape == "slab":
        inside = np.broadcast_to(np.abs(x) <= ax, (nz, ny, nx))
    else:
        raise ValueError(f"unknown bulk shape {shape!r}")
    return np.where(inside, MASK_SC, MASK_OUT).astype(np.uint8)


def _distance_inside(mask: np.ndarray, spacing: tuple[float, ...]) -> np.ndarray:
    """Euclidean distance from each conductor cell centre to the nearest free-space cell centre."""
    from scipy.ndimage import distance_transform_edt
    return distance_transform_edt(mask != MASK_OUT, sampling=spacing)


def _smooth_noise(r: np.random.Generator, shape: tuple[int, ...], modes: int = 4) -> np.ndarray:
    """Sum of a few low-frequency cosines with seeded amplitudes and phases, max |.| <= 1."""
    out = np.zeros(shape)
    grids = np.meshgrid(*[np.arange(s) / s for s in shape], indexing="ij")
    for _ in range(modes):
        k = [int(r.integers(1, 4)) for _ in shape]
        ph = r.uniform(0, 2 * np.pi)
        arg = sum(2 * np.pi * kk * g for kk, g in zip(k, grids))
        out += r.uniform(-1, 1) * np.cos(arg + ph)
    return out / max(1.0, np.abs(out).max())


def film_state(mask: np.ndarray, Lx: float, Ly: float, seed: int, *,
               amplitude: float = 1.0, depth: float = 0.3, noise: float = 0.1) -> np.ndarray:
    """A plausible stream function g (ny, nx): zero on free space, a critical-state 'sand pile'
    min(distance to the edge, depth) inside, times (1 + noise * smooth random field)."""
    ny, nx = mask.shape
    d = _distance_inside(mask, (2 * Ly / ny, 2 * Lx / nx))
    r = rng(seed)
    g = amplitude * np.minimum(d, depth) * (1.0 + noise * _smooth_noise(r, mask.shape))
    return np.where(mask != MASK_OUT, g, 0.0)


def bulk_state(mask: np.ndarray, L: tuple[float, float, float], seed: int, *,
               h0: float = 0.2, depth: float = 0.15, noise: float = 0.05) -> np.ndarray:
    """A plausible field h (3, nz, ny, nx): h_z = h0 - min(distance, depth) inside the
    conductor (a shielding profile with |grad h_z| ~ 1), h0 outside, plus small smooth noise
    in all three components."""
    nz, ny, nx = mask.shape
    Lx, Ly, Lz = L
    d = _distance_inside(mask, (2 * Lz / nz, 2 * Ly / ny, 2 * Lx / nx))
    r = rng(seed)
    h = np.zeros((3,) + mask.shape)
    h[2] = h0 - np.minimum(d, depth)
    for c in range(3):
        h[c] += noise * _smooth_noise(r, mask.shape)
    return h


def jc_map_lognormal(shape: tuple[int, ...], seed: int, sigma: float = 0.2) -> np.ndarray:
    """Per-cell critical current density exp(sigma z - sigma^2/2), z ~ N(0,1) i.i.d."""
    z = rng(seed).standard_normal(shape)
    return np.exp(sigma * z - 0.5 * sigma * sigma)


# --------------------------------------------------------------------------------------------
# standard workloads (sizes and parameters of the published configurations)
# --------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    dim: int
    nx: int
    ny: int
    nz: int
    Lx: float
    Ly: float
    Lz: float
    mask: np.ndarray
    n: float
    rho_out: float
    precision: int               # 0 = FP64 transforms, 1 = FP32 transforms with FP64 state
    t0: float
    t1: float
    he_knots: tuple[tuple[float, ...], tuple[float, ...]] | None = None
    he_sin: tuple[float, float] | None = None      # (amplitude, period)
    sigma: float = 0.0                              # <= 0: sqrt(sum dx^2)
    lam: float = 0.7
    iter_tol: float = 2e-4
    iter_max: int = 3000          # a cold start (t = 0, g = 0) needs ~700 iterations at 128^2
    rtol: float = 1e-6
    atol: float = 1e-6
    jc: float = 1.0
    jc_map: np.ndarray | None = None
    vector_he: tuple[float, float, float] = (0.0, 0.0, 1.0)
    gamma: float = 1.0            # elliptic anisotropy of the law (film: along y, bulk: along z)
    b0: float = 0.0               # bulk Kim-type jc / (1 + |h|/b0); 0: none


def square_film_128(precision: int = 0) -> Workload:
    """Square film Omega=[-1,1]^2 (64x64 cells) centred in a 128x128 periodic grid, D=[-2,2]^2,
    n=19, h_e ramped linearly 0 -> 0.5 over t in [0,1], rtol=atol=1e-6."""
    nx = ny = 128
    L = 2.0
    m = film_mask(nx, ny, L, L, "rect", ax=1.0, ay=1.0)
    return Workload("square_film_64_in_128_fp64" if precision == 0 else "square_film_64_in_128_fp32",
                    2, nx, ny, 1, L, L, 0.0, m, n=19.0, rho_out=1.0, precision=precision,
                    t0=0.0, t1=1.0, he_knots=((0.0, 1.0), (0.0, 0.5)))


def rect_film_2048(precision: int = 1, n_grid: int = 2048) -> Workload:
    """Rectangular film 1024x512 cells (aspect 2:1), Omega=[-1,1]x[-1/2,1/2], in a 2048x2048
    periodic grid with D=[-2,2]^2, n=30, one sinusoidal cycle h_e = 0.8 sin(2 pi t), t in [0,1].
    `n_grid` rescales the grid (cells per unit length scale with it)."""
    L = 2.0
    m = film_mask(n_grid, n_grid, L, L, "rect", ax=1.0, ay=0.5)
    return Workload(f"rect_film_{n_grid // 2}x{n_grid // 4}_in_{n_grid}sq", 2, n_grid, n_grid, 1,
                    L, L, 0.0, m, n=30.0, rho_out=1.0, precision=precision, t0=0.0, t1=1.0,
                    he_sin=(0.8, 1.0))


def cube_bulk(n_grid: int = 128, precision: int = 1) -> Workload:
    """Cube Omega=[-1/2,1/2]^3 (n_grid/2 cells per side) in an n_grid^3 periodic grid with
    D=[-1,1]^3, n=25, rho_out=5, delta_it=1e-4, h_e,z ramped 0 -> 0.25 on [0,0.5], then held."""
    L = 1.0
    m = bulk_mask(n_grid, n_grid, n_grid, L, L, L, "box", ax=0.5, ay=0.5, az=0.5)
    return Workload(f"cube_{n_grid // 2}_in_{n_grid}cubed", 3, n_grid, n_grid, n_grid, L, L, L, m,
                    n=25.0, rho_out=5.0, precision=precision, t0=0.0, t1=1.0,
                    he_knots=((0.0, 0.5, 1.0), (0.0, 0.25, 0.25)), iter_tol=1e-4)



def adjoint_film(n_grid: int = 1024, precision: int = 1, T: float = 0.1, knots: int = 16,
                 jc_seed: int = 5) -> Workload:
    """The film of the gradient (adjoint) workload: a square film of n_grid/2 cells per side,
    Omega = [-1,1]^2, in an n_grid^2 periodic grid with D = [-2,2]^2, n = 30, a per-cell critical
    current density exp(0.2 z - 0.02), z ~ N(0,1) i.i.d. (seed jc_seed), and h_e(t) piecewise
    linear through `knots` knots evenly spaced on [0, T] with the baseline values 0.5 t / T."""
    L = 2.0
    m = film_mask(n_grid, n_grid, L, L, "rect", ax=1.0, ay=1.0)
    kt = tuple(float(x) for x in np.linspace(0.0, T, knots))
    kv = tuple(0.5 * t / T for t in kt)
    wl = Workload(f"square_film_{n_grid // 2}_in_{n_grid}_adjoint", 2, n_grid, n_grid, 1, L, L, 0.0,
                  m, n=30.0, rho_out=1.0, precision=precision, t0=0.0, t1=T, he_knots=(kt, kv))
    wl.jc_map = jc_map_lognormal((n_grid, n_grid), seed=jc_seed, sigma=0.2)
    return wl


def segment_steps(knot_times, n_steps: int) -> list[tuple[float, float]]:
    """n_steps (t, h) steps covering [t_0, t_last] of the knots, spread as evenly as whole numbers
    allow over the segments and uniform inside each, so that no step crosses a knot."""
    kt = [float(t) for t in knot_times]
    nseg = len(kt) - 1
    per = [n_steps // nseg + (1 if k < n_steps % nseg else 0) for k in range(nseg)]
    steps = []
    for k in range(nseg):
        h = (kt[k + 1] - kt[k]) / per[k]
        steps += [(kt[k] + i * h, h) for i in range(per[k])]
    return steps


def film_batch(count: int = 256, seed: int = 3, max_side: int = 512, precision: int = 1) -> list[Workload]:
    """Independent films of a parameter/geometry sweep: the shape class is uniform over
    {square, rectangle with aspect U[1, 2], disk}, the film side s (cells) over 64 .. max_side,
    the power n over {19, 30, 50} and the ramp amplitude (h_e from 0 to it over [0, 1]) over
    U[0.2, 1].  The film's long side spans [-1, 1] with s cells; the periodic grid is the next
    power of two >= 2 s cells per axis (at least twice the film, as the paper's examples),
    D = [-L, L]^2 with L = grid / s.""" 
    r = rng(seed)
    out = []
    for i in range(count):
        cls = int(r.integers(0, 3))
        s = int(r.integers(64, max_side + 1))
        n = float((19.0, 30.0, 50.0)[int(r.integers(0, 3))])
        amp = float(r.uniform(0.2, 1.0))
        aspect = float(r.uniform(1.0, 2.0))
        grid = 1 << int(np.ceil(np.log2(2 * s)))
        L = 2.0 * grid / (2 * s)            # film long half-side 1 with s cells across it
        if cls == 0:
            m, name = film_mask(grid, grid, L, L, "rect", ax=1.0, ay=1.0), "square"
        elif cls == 1:
            m, name = film_mask(grid, grid, L, L, "rect", ax=1.0, ay=1.0 / aspect), "rect"
        else:
            m, name = film_mask(grid, grid, L, L, "disk", radius=1.0), "disk"
        out.append(Workload(f"batch{seed}_{i}_{name}_{s}_in_{grid}", 2, grid, grid, 1, L, L, 0.0, m,
                            n=n, rho_out=1.0, precision=precision, t0=0.0, t1=1.0,
                            he_knots=((0.0, 1.0), (0.0, amp)), rtol=1e-3, atol=1e-6))
    return out
