"""Grid, permittivity and FDFD operator (oracle; test infrastructure only).

The paper leaves the Maxwell operator abstract ("A is the Maxwell operator ... a
finite-difference ... discretization", Sec. 4.1).  The reading used here: the 2-D
scalar Helmholtz equation for E_z (or H_z in a homogeneous-epsilon reading) at
wavelength 1 on a uniform grid of spacing h, with a stretched-coordinate PML on
all four sides, multiplied through by s_x s_y so that the matrix is complex
symmetric (A = A^T):

  s_y^j/h^2 [ (u_{i+1,j}-u_{ij})/s_x^{i+1/2} - (u_{ij}-u_{i-1,j})/s_x^{i-1/2} ]
+ s_x^i/h^2 [ (u_{i,j+1}-u_{ij})/s_y^{j+1/2} - (u_{ij}-u_{i,j-1})/s_y^{j-1/2} ]
+ k0^2 eps_ij s_x^i s_y^j u_ij  =  b_ij ,        u = 0 outside the grid.

Unknown order k = i*ny + j (column-major in x): block-tridiagonal along x.
Node (i, j) sits at x_i = (i - npml + 1/2) h, y_j = (j + 1/2) h.
Interior columns S = {npml <= i < nx - npml}; n_src = |S|.
Time convention exp(-i omega t); outgoing waves exp(+i k r).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from workloads import (GridDesc, Objective, OBJ_POINT, OBJ_PLANEWAVE,
                       OBJ_VIRTUAL_FOCUS, OBJ_USER_ROW)


class Grid:
    """Derived geometry of a GridDesc (all plain arithmetic on the description)."""

    def __init__(self, d: GridDesc):
        self.d = d
        self.h = 1.0 / d.ppl
        self.k0 = 2.0 * math.pi
        self.nx = d.n_cells * d.cell_px + 2 * d.npml
        self.ny = d.ny
        self.npml = d.npml
        self.n_src = self.nx - 2 * d.npml
        self.width = self.n_src * self.h
        self.j_src = d.npml + d.src_offset
        self.j_pillar0 = d.npml + d.rows_sub
        self.j_pillar1 = self.j_pillar0 + d.rows_pillar
        self.rows_air = d.ny - 2 * d.npml - d.rows_sub - d.rows_pillar
        if self.rows_air < 1:
            raise ValueError("grid too short: no air rows above the pillars")
        self.N = self.nx * self.ny
        self.k_sub = self.k0 * math.sqrt(d.eps_sub)

    # coordinates ---------------------------------------------------------------
    def x(self, i):
        return (np.asarray(i, dtype=np.float64) - self.npml + 0.5) * self.h

    def x_src(self):
        """Abscissae of the interior columns S (the source / cross-correlation plane)."""
        return self.x(np.arange(self.npml, self.nx - self.npml))

    # PML ---------------------------------------------------------------------------
    def _sigma(self, xi):
        d = self.npml * self.h
        m = self.d.pml_m
        smax = -(m + 1) * math.log(self.d.pml_R0) / (2.0 * d)
        xi = np.clip(xi, 0.0, None)
        return smax * (xi / d) ** m

    def _stretch(self, depth):
        return 1.0 + 1j * self._sigma(depth) / self.k0

    def pml(self):
        """s_x at nodes (nx), s_x at half nodes x_{i-1/2} for i = 0..nx (nx+1),
        s_y at nodes (ny), s_y at half nodes y_{j-1/2} for j = 0..ny (ny+1)."""
        h, W = self.h, self.width
        xn = self.x(np.arange(self.nx))
        xh = (np.arange(self.nx + 1) - self.npml) * h
        yn = (np.arange(self.ny) + 0.5) * h
        yh = np.arange(self.ny + 1) * h
        y0, y1 = self.npml * h, (self.ny - self.npml) * h
        depth_x = lambda x: np.maximum(np.maximum(-x, x - W), 0.0)
        depth_y = lambda y: np.maximum(np.maximum(y0 - y, y - y1), 0.0)
        return (self._stretch(depth_x(xn)), self._stretch(depth_x(xh)),
                self._stretch(depth_y(yn)), self._stretch(depth_y(yh)))


def rasterize_eps(g: Grid, widths: np.ndarray) -> np.ndarray:
    """eps[i, j] (nx, ny).  Pillar m is centred in unit cell m at x = (m + 1/2) p;
    in the pillar rows each grid column takes the area-weighted average of the
    pillar and air permittivities over its extent [x_i - h/2, x_i + h/2] (the two
    pillars that may share a column both count).  Substrate below, air above."""
    d = g.d
    widths = np.asarray(widths, dtype=np.float64)
    if widths.shape != (d.n_cells,):
        raise ValueError("need one width per cell")
    p = d.cell_px * g.h
    eps = np.empty((g.nx, g.ny))
    eps[:, : g.j_pillar0] = d.eps_sub
    eps[:, g.j_pillar0:] = d.eps_air
    frac = np.zeros(g.nx)
    for i in range(g.nx):
        lo, hi = g.x(i) - g.h / 2, g.x(i) + g.h / 2
        m0 = max(int(math.floor(lo / p)) - 1, 0)
        m1 = min(int(math.floor(hi / p)) + 1, d.n_cells - 1)
        acc = 0.0
        for m in range(m0, m1 + 1):
            c = (m + 0.5) * p
            a, b = c - widths[m] / 2, c + widths[m] / 2
            acc += max(0.0, min(hi, b) - max(lo, a))
        frac[i] = acc / g.h
    eps[:, g.j_pillar0:g.j_pillar1] = (d.eps_air + frac * (d.eps_pillar - d.eps_air))[:, None]
    return eps


def stencil_coefficients(g: Grid, eps: np.ndarray):
    """The five stencil coefficient arrays of A.

    Returns (diag[nx, ny], cxp[nx-1, ny], cyp[nx, ny-1]) where cxp[i, j] couples
    (i, j) and (i+1, j) and cyp[i, j] couples (i, j) and (i, j+1); A is symmetric
    so the same values couple in the other direction."""
    sx, sxh, sy, syh = g.pml()
    h2 = g.h * g.h
    SX = sx[:, None]
    SY = sy[None, :]
    inv_sxh = 1.0 / sxh
    inv_syh = 1.0 / syh
    diag = (-SY / h2 * (inv_sxh[1:, None] + inv_sxh[:-1, None])
            - SX / h2 * (inv_syh[None, 1:] + inv_syh[None, :-1])
            + g.k0 ** 2 * eps * SX * SY)
    cxp = SY / h2 * inv_sxh[1:-1, None]            # s_y^j / (h^2 s_x^{i+1/2}), i = 0..nx-2
    cyp = SX / h2 * inv_syh[None, 1:-1]            # s_x^i / (h^2 s_y^{j+1/2}), j = 0..ny-2
    return diag, np.broadcast_to(cxp, (g.nx - 1, g.ny)).copy(), cyp


def assemble(g: Grid, eps: np.ndarray) -> sp.csc_matrix:
    """Sparse A (N x N, complex128) in the unknown order k = i*ny + j."""
    diag, cxp, cyp = stencil_coefficients(g, eps)
    nx, ny = g.nx, g.ny
    k = np.arange(g.N).reshape(nx, ny)
    rows = [k.ravel(), k[:-1].ravel(), k[1:].ravel(), k[:, :-1].ravel(), k[:, 1:].ravel()]
    cols = [k.ravel(), k[1:].ravel(), k[:-1].ravel(), k[:, 1:].ravel(), k[:, :-1].ravel()]
    vals = [diag.ravel(), cxp.ravel(), cxp.ravel(), cyp.ravel(), cyp.ravel()]
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(g.N, g.N))


def apply_A(g: Grid, coeffs, u: np.ndarray) -> np.ndarray:
    """A u by the stencil (u as an (nx, ny) array)."""
    diag, cxp, cyp = coeffs
    out = diag * u
    out[:-1] += cxp * u[1:]
    out[1:] += cxp * u[:-1]
    out[:, :-1] += cyp * u[:, 1:]
    out[:, 1:] += cyp * u[:, :-1]
    return out


# ---- sources and objectives -----------------------------------------------------

def planewave_source(g: Grid, theta: float) -> np.ndarray:
    """Equivalent current b0(theta) of a unit-power planewave incident at angle theta
    (measured in the substrate), Sec. 4.1: a line current on the source row over the
    interior columns, amplitude sqrt(cos theta) (unit power), phase exp(i k_s sin(theta) x)."""
    b = np.zeros((g.nx, g.ny), dtype=np.complex128)
    xs = g.x_src()
    b[g.npml:g.nx - g.npml, g.j_src] = math.sqrt(math.cos(theta)) * np.exp(
        1j * g.k_sub * math.sin(theta) * xs)
    return b


def objective_vector(g: Grid, obj: Objective) -> np.ndarray:
    """w (nx, ny) such that the figure of merit is |w^dag u|^2 (Sec. 4.1)."""
    w = np.zeros((g.nx, g.ny), dtype=np.complex128)
    if obj.kind == OBJ_POINT:
        if not (0 <= obj.i_f < g.nx and 0 <= obj.j_f < g.ny):
            raise ValueError("focus outside the grid")
        w[obj.i_f, obj.j_f] = 1.0
        return w
    j = obj.monitor_row
    if not (0 <= j < g.ny):
        raise ValueError("monitor row outside the grid")
    xs = g.x_src()
    if obj.kind == OBJ_PLANEWAVE:
        w[g.npml:g.nx - g.npml, j] = np.exp(1j * g.k0 * math.sin(obj.theta_out) * xs)
    elif obj.kind == OBJ_VIRTUAL_FOCUS:
        K = virtual_focus_kernel(g, obj.x_f - xs, obj.d_rows)
        w[g.npml:g.nx - g.npml, j] = np.conj(K)
    elif obj.kind == OBJ_USER_ROW:
        row = np.asarray(obj.w_row, dtype=np.complex128)
        if row.shape != (g.n_src,):
            raise ValueError("w_row must have n_src entries")
        w[g.npml:g.nx - g.npml, j] = row
    else:
        raise ValueError("unknown objective kind")
    return w


def _gl_unit(n: int):
    """Gauss-Legendre nodes/weights on [-1, 1] from oracle.light (Newton on the
    three-term recurrence)."""
    from oracle.light import gauss_legendre
    return gauss_legendre(n)


def virtual_focus_kernel(g: Grid, delta: np.ndarray, d_rows: int,
                         panels: int = 256, order: int = 32) -> np.ndarray:
    """Lattice propagator K(Delta) from a row of homogeneous air to the point d_rows
    rows above it, horizontal offset Delta, for a field with no sources above the row
    (outgoing upward).  On the infinite lattice,

        u(x_f, j_m + D) = sum_i K(x_f - x_i) u(x_i, j_m),
        K(Delta) = (h/pi) int_0^{pi/h} exp(i q(k) D) cos(k Delta) dk,
        cos q = 2 - cos(k h) - k0^2 h^2 eps_air / 2,  q >= 0 (propagating) or q = i alpha.

    Composite Gauss-Legendre in t with k = k_c -+ t^2 on each side of the branch point
    k_c (where q = 0), which makes the integrand smooth."""
    h, k0, D = g.h, g.k0, int(d_rows)
    ea = g.d.eps_air
    delta = np.asarray(delta, dtype=np.float64)
    kc = math.acos(1.0 - k0 * k0 * h * h * ea / 2.0) / h
    kmax = math.pi / h
    xg, wg = _gl_unit(order)

    def composite(a, b):
        edges = np.linspace(a, b, panels + 1)
        mid = 0.5 * (edges[1:] + edges[:-1])
        half = 0.5 * (edges[1:] - edges[:-1])
        t = (mid[:, None] + half[:, None] * xg[None, :]).ravel()
        wt = (half[:, None] * wg[None, :]).ravel()
        return t, wt

    out = np.zeros(delta.shape, dtype=np.complex128)
    # propagating side: k = kc - t^2, t in [0, sqrt(kc)], dk = 2 t dt
    t, wt = composite(0.0, math.sqrt(kc))
    k = kc - t * t
    cq = 2.0 - np.cos(k * h) - k0 * k0 * h * h * ea / 2.0
    q = np.arccos(np.clip(cq, -1.0, 1.0))
    phase = np.exp(1j * q * D) * (2.0 * t * wt)
    # evanescent side: k = kc + t^2, t in [0, sqrt(kmax - kc)]
    t2, wt2 = composite(0.0, math.sqrt(kmax - kc))
    k2 = kc + t2 * t2
    cq2 = 2.0 - np.cos(k2 * h) - k0 * k0 * h * h * ea / 2.0
    alpha = np.arccosh(np.maximum(cq2, 1.0))
    decay = np.exp(-alpha * D) * (2.0 * t2 * wt2)
    flat = delta.ravel()
    res = np.empty(flat.shape, dtype=np.complex128)
    for s in range(0, flat.size, 256):
        dl = flat[s:s + 256]
        res[s:s + 256] = (np.cos(np.outer(dl, k)) @ phase
                          + np.cos(np.outer(dl, k2)) @ decay)
    out = (h / math.pi) * res.reshape(delta.shape)
    return out
