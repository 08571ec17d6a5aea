"""Seeded synthetic workloads for the reciprocal incoherent-light evaluation.

This module only *describes* problems: grid parameters, pillar widths drawn from a
seed, and the light / objective parameters of each workload.  It holds none of the
method's arithmetic.  The CUDA library and the CPU oracle each derive every grid
quantity (nx, ny, coordinates, PML, permittivity, operator) from these descriptions
on their own.

Units: wavelength lambda = 1.  Angles in radians.

Workloads (sizes follow the problem statement of each case):
  c1_concentrator  50 cells  (20 lambda wide), nx = 440,   ny = 128, on-grid focus
                   3 lambda above the pillars, light uniform on +-20 deg,
                   brute force over 201 angles.
  c2_collimator    500 cells (200 lambda wide), nx = 4040, ny = 160, output angle 0,
                   annular light 10..30 deg, brute force over 1000 angles.
  c3_precision     2500 cells (1000 lambda), nx = 20040, ny = 224, virtual focus
                   50 lambda above the monitor row, light +-20 deg.
  c4_gradient      c2 geometry, virtual focus 20 lambda, light +-15 deg.
  tiny / small     reduced grids for fast tests (thinner PML, fewer rows).
  serving_requests a stream of requests with Poisson arrivals: width log-uniform in
                   20..500 lambda (50..1250 cells, ny = 160), concentrator (virtual focus
                   5..20 lambda up) or collimator (output angle 0..10 deg) half and half,
                   light a cone (half-angle 5..40 deg) or an annulus (inner 5..20 deg,
                   outer inner + 5..20 deg) half and half, 30 % also asking for the
                   gradient.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---- enumerations shared by the C-ABI and the oracle (plain integers) -------------
OBJ_POINT = 0          # concentrator, focus on a grid node: w = e_f
OBJ_PLANEWAVE = 1      # collimator: w = planewave at the output angle on the monitor row
OBJ_VIRTUAL_FOCUS = 2  # concentrator, focus d rows above the monitor row (homogeneous air)
OBJ_USER_ROW = 3       # caller-supplied w on the monitor row

LIGHT_CONE = 0         # uniform in theta on [-c, c]
LIGHT_ANNULUS = 1      # uniform in theta on [th1, th2] U [-th2, -th1]
LIGHT_USER_LAGS = 2    # caller-supplied real, even W(m h), m = 0..n_src-1
LIGHT_TABULATED = 3    # rho given at angles 0 <= theta_0 < ... < pi/2, piecewise linear, even

PREC_FP64 = 0
PREC_FP32_REFINE = 1


@dataclasses.dataclass
class GridDesc:
    """Problem geometry.  All lengths in wavelengths; rows/columns in grid cells."""
    n_cells: int
    ny: int
    ppl: int = 20              # grid points per wavelength (h = 1/ppl)
    cell_px: int = 8           # unit-cell period in grid cells (0.4 lambda at 20 px/lambda)
    npml: int = 20             # PML thickness in cells, all four sides
    rows_sub: int = 12         # substrate rows between the bottom PML and the pillars
    rows_pillar: int = 12      # pillar height in rows (0.6 lambda)
    src_offset: int = 2        # source row = npml + src_offset (inside the substrate)
    eps_pillar: float = 5.3
    eps_sub: float = 2.1
    eps_air: float = 1.0
    pml_R0: float = 1e-8
    pml_m: int = 3
    prec: int = PREC_FP64


@dataclasses.dataclass
class Objective:
    kind: int
    monitor_row: int = -1      # row of the objective vector (OBJ_PLANEWAVE / VIRTUAL / USER)
    i_f: int = 0               # OBJ_POINT: focus node
    j_f: int = 0
    theta_out: float = 0.0     # OBJ_PLANEWAVE: output angle in air
    x_f: float = 0.0           # OBJ_VIRTUAL_FOCUS: focus abscissa (lambda)
    d_rows: int = 0            # OBJ_VIRTUAL_FOCUS: focus height above the monitor row, in rows
    w_row: np.ndarray | None = None   # OBJ_USER_ROW: complex128[n_src]


@dataclasses.dataclass
class Light:
    kind: int
    c: float = 0.0
    th1: float = 0.0
    th2: float = 0.0
    lags: np.ndarray | None = None    # LIGHT_USER_LAGS: float64[n_src]
    theta: np.ndarray | None = None   # LIGHT_TABULATED: nodes (radians, ascending, in [0, pi/2))
    rho: np.ndarray | None = None     # LIGHT_TABULATED: density at the nodes (>= 0)


@dataclasses.dataclass
class Workload:
    name: str
    grid: GridDesc
    objective: Objective
    light: Light
    n_angles: int              # brute-force quadrature points
    seed: int = 0


def widths(n_cells: int, seed: int, lo: float = 0.08, hi: float = 0.36) -> np.ndarray:
    """Pillar widths (lambda), i.i.d. uniform on [lo, hi], from a seeded generator."""
    return np.random.default_rng(seed).uniform(lo, hi, n_cells)


def _pillar_top(g: GridDesc) -> int:
    return g.npml + g.rows_sub + g.rows_pillar


def deg(x: float) -> float:
    return x * math.pi / 180.0


def c1_concentrator(seed: int = 0) -> Workload:
    g = GridDesc(n_cells=50, ny=128)
    nx = g.n_cells * g.cell_px + 2 * g.npml
    top = _pillar_top(g)
    obj = Objective(kind=OBJ_POINT, i_f=nx // 2, j_f=top + 3 * g.ppl)
    return Workload("c1_concentrator", g, obj, Light(LIGHT_CONE, c=deg(20)), 201, seed)


def c2_collimator(seed: int = 0) -> Workload:
    g = GridDesc(n_cells=500, ny=160)
    obj = Objective(kind=OBJ_PLANEWAVE, monitor_row=_pillar_top(g) + 10, theta_out=0.0)
    return Workload("c2_collimator", g, obj,
                    Light(LIGHT_ANNULUS, th1=deg(10), th2=deg(30)), 1000, seed)


def c3_precision(seed: int = 0) -> Workload:
    g = GridDesc(n_cells=2500, ny=224, prec=PREC_FP32_REFINE)
    width = g.n_cells * g.cell_px / g.ppl
    mrow = _pillar_top(g) + 10
    obj = Objective(kind=OBJ_VIRTUAL_FOCUS, monitor_row=mrow, x_f=width / 2,
                    d_rows=50 * g.ppl - 10)
    return Workload("c3_precision", g, obj, Light(LIGHT_CONE, c=deg(20)), 0, seed)


def c4_gradient(seed: int = 0) -> Workload:
    g = GridDesc(n_cells=500, ny=160)
    width = g.n_cells * g.cell_px / g.ppl
    mrow = _pillar_top(g) + 10
    obj = Objective(kind=OBJ_VIRTUAL_FOCUS, monitor_row=mrow, x_f=width / 2,
                    d_rows=20 * g.ppl - 10)
    return Workload("c4_gradient", g, obj, Light(LIGHT_CONE, c=deg(15)), 0, seed)


def tiny(seed: int = 0, n_cells: int = 3, ny: int = 48, kind: int = OBJ_POINT) -> Workload:
    """A grid small enough for dense linear algebra (nx = 8 n_cells + 16)."""
    g = GridDesc(n_cells=n_cells, ny=ny, npml=8, rows_sub=6, rows_pillar=6)
    nx = g.n_cells * g.cell_px + 2 * g.npml
    top = _pillar_top(g)
    if kind == OBJ_POINT:
        obj = Objective(kind=OBJ_POINT, i_f=nx // 2, j_f=top + 8)
    elif kind == OBJ_PLANEWAVE:
        obj = Objective(kind=OBJ_PLANEWAVE, monitor_row=top + 4, theta_out=deg(5))
    else:
        obj = Objective(kind=OBJ_VIRTUAL_FOCUS, monitor_row=top + 4,
                        x_f=n_cells * g.cell_px / g.ppl / 2, d_rows=20)
    return Workload("tiny", g, obj, Light(LIGHT_CONE, c=deg(20)), 64, seed)


def small(seed: int = 0, n_cells: int = 12, ny: int = 64, kind: int = OBJ_PLANEWAVE) -> Workload:
    """A few-thousand-unknown grid that still spans several BCR levels."""
    g = GridDesc(n_cells=n_cells, ny=ny, npml=10, rows_sub=8, rows_pillar=12)
    nx = g.n_cells * g.cell_px + 2 * g.npml
    top = _pillar_top(g)
    if kind == OBJ_POINT:
        obj = Objective(kind=OBJ_POINT, i_f=nx // 2, j_f=top + 20)
    elif kind == OBJ_PLANEWAVE:
        obj = Objective(kind=OBJ_PLANEWAVE, monitor_row=top + 6, theta_out=deg(3))
    else:
        obj = Objective(kind=OBJ_VIRTUAL_FOCUS, monitor_row=top + 6,
                        x_f=n_cells * g.cell_px / g.ppl / 2, d_rows=40)
    return Workload("small", g, obj, Light(LIGHT_ANNULUS, th1=deg(10), th2=deg(30)), 128, seed)


@dataclasses.dataclass
class Request:
    arrival_s: float           # seconds after the start of the stream
    grid: GridDesc
    widths: np.ndarray
    objective: Objective
    light: Light
    want_grad: bool
    seed: int
    design_key: int = 0        # != 0: the server may keep the factorisation for a later request


def serving_requests(n: int, rate_per_s: float, seed: int = 0, cells=(50, 1250), ny: int = 160,
                     grad_fraction: float = 0.3, prec: int = PREC_FP32_REFINE,
                     repeat_fraction: float = 0.0) -> list:
    """n requests with exponential inter-arrival times (mean 1/rate), each a seeded
    metasurface of its own (design seed = seed * 1_000_003 + k).

    With repeat_fraction > 0 every design carries a key (its seed + 1), and that fraction of
    the requests (after the first) re-evaluate one of the last 32 designs -- same grid,
    widths, objective and key -- under a new angular distribution, as a designer comparing
    light sources on one metasurface would."""
    rng = np.random.default_rng(seed)
    rep = np.random.default_rng(seed + 7_777_777)
    out = []
    t = 0.0
    lo, hi = math.log(cells[0]), math.log(cells[1])
    for k in range(n):
        t += rng.exponential(1.0 / rate_per_s) if rate_per_s > 0 else 0.0
        if repeat_fraction > 0 and out and rep.uniform() < repeat_fraction:
            src = out[-1 - int(rep.integers(0, min(32, len(out))))]
            th1 = rep.uniform(5.0, 20.0)
            light = Light(LIGHT_ANNULUS, th1=deg(th1), th2=deg(th1 + rep.uniform(5.0, 20.0)))
            out.append(Request(t, src.grid, src.widths, src.objective, light,
                               bool(rep.uniform() < grad_fraction), src.seed, src.design_key))
            continue
        nc = int(round(math.exp(rng.uniform(lo, hi))))
        g = GridDesc(n_cells=nc, ny=ny, prec=prec)
        top = _pillar_top(g)
        if rng.uniform() < 0.5:
            width = nc * g.cell_px / g.ppl
            obj = Objective(kind=OBJ_VIRTUAL_FOCUS, monitor_row=top + 10, x_f=width / 2,
                            d_rows=int(round(rng.uniform(5.0, 20.0) * g.ppl)))
        else:
            obj = Objective(kind=OBJ_PLANEWAVE, monitor_row=top + 10,
                            theta_out=deg(rng.uniform(0.0, 10.0)))
        if rng.uniform() < 0.5:
            light = Light(LIGHT_CONE, c=deg(rng.uniform(5.0, 40.0)))
        else:
            th1 = rng.uniform(5.0, 20.0)
            light = Light(LIGHT_ANNULUS, th1=deg(th1), th2=deg(th1 + rng.uniform(5.0, 20.0)))
        dseed = seed * 1_000_003 + k
        out.append(Request(t, g, widths(nc, dseed), obj, light,
                           bool(rng.uniform() < grad_fraction), dseed,
                           dseed + 1 if repeat_fraction > 0 else 0))
    return out


WORKLOADS = {
    "c1_concentrator": c1_concentrator,
    "c2_collimator": c2_collimator,
    "c3_precision": c3_precision,
    "c4_gradient": c4_gradient,
}
