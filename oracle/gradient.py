"""Gradient of the averaged figure of merit with respect to the pillar widths
(oracle; test infrastructure only).

Adjoint form (Sec. 4.1, the paragraph after Eq. 7: the gradient of v^dag W v is
2 Re(v^dag W dv), and dv needs one more solve with the same matrix).  With
z = A^{-1} conj(w) and v = conj(z) on the source plane S (row j_src):

    F = v^dag W v,   dF = 2 Re(v^dag W dv) = 2 Re(g^T dz_S),   g = W v ,

because W is real and symmetric.  dz = -A^{-1} (dA) z, and A = A^T, so with the
adjoint field mu = A^{-1} P_S^T g (g placed on row j_src over S, zero elsewhere):

    dF = -2 Re( mu^T (dA) z ) = -2 Re sum_c mu_c z_c (dA)_cc .

Only the diagonal of A depends on the design: (dA)_cc = k0^2 s_x s_y d(eps_c), and
eps = eps_air + f (eps_pillar - eps_air) in the pillar rows, f the area fill of the
column (see oracle.grid.rasterize_eps).  The fill is piecewise linear in each width:
moving one edge of pillar m by dw/2 changes the fill of the column holding that edge
by dw/(2h).  At a tie (edge exactly on a column boundary) the derivative taken is the
one for a growing width: the right edge b counts in the column with lo <= b < hi,
the left edge a in the column with lo < a <= hi.

Brute-force form (Eq. 6 differentiated angle by angle), used to pin the adjoint:
with u_q = A^{-1} b0(theta_q), a_q = w^dag u_q, c_q = Omega_q rho(theta_q),

    dF_bf = sum_q c_q 2 Re( conj(a_q) w^dag du_q ),   w^dag du_q = -sum_c z_c (dA)_cc u_{q,c}

(w^dag A^{-1} = z^T since A is symmetric).  For a rule symmetric in theta, F_bf equals
v^dag W_N v exactly with the Toeplitz lags W_N(D) = sum_q c_q cos(theta_q)
cos(k_s sin(theta_q) D), so the two gradients agree to rounding.
"""
from __future__ import annotations

import math

import numpy as np

from oracle.grid import Grid, planewave_source
from oracle.reciprocal import Evaluation, reciprocal_field, source_plane


def fill_derivative(g: Grid, widths: np.ndarray) -> np.ndarray:
    """d f_i / d w_m as a dense (nx, n_cells) array, from the area-fill definition
    column by column (same column bounds as the raster)."""
    d = g.d
    widths = np.asarray(widths, dtype=np.float64)
    p = d.cell_px * g.h
    D = np.zeros((g.nx, d.n_cells))
    for i in range(g.nx):
        lo, hi = g.x(i) - g.h / 2, g.x(i) + g.h / 2
        for m in range(d.n_cells):
            c = (m + 0.5) * p
            a, b = c - widths[m] / 2, c + widths[m] / 2
            if lo <= b < hi:
                D[i, m] += 0.5 / g.h
            if lo < a <= hi:
                D[i, m] += 0.5 / g.h
    return D


def toeplitz_apply(lags: np.ndarray, v: np.ndarray) -> np.ndarray:
    """(W v)_i = sum_l W_{|i-l|} v_l with the full Toeplitz matrix formed explicitly."""
    n = v.size
    idx = np.arange(n)
    T = lags[np.abs(idx[:, None] - idx[None, :])]
    return T @ v


def _design_diag_weight(g: Grid) -> np.ndarray:
    """k0^2 s_x s_y over the whole grid: d(A_cc)/d(eps_c)."""
    sx, _, sy, _ = g.pml()
    return g.k0 ** 2 * sx[:, None] * sy[None, :]


def _to_widths(g: Grid, dF_deps_col: np.ndarray, widths: np.ndarray) -> np.ndarray:
    """Chain rule from dF/d(fill of pillar-row column i) to dF/dw_m."""
    d = g.d
    return fill_derivative(g, widths).T @ (dF_deps_col * (d.eps_pillar - d.eps_air))


def avg_intensity_grad(ev: Evaluation, widths: np.ndarray, lags: np.ndarray | None = None):
    """(F, dF/dwidths, z, mu) by the adjoint method on one factorisation."""
    g = ev.g
    if lags is None:
        lags = ev.lags()
    z = ev.solver.solve(np.conj(ev.w))
    v = source_plane(g, np.conj(z))
    gv = toeplitz_apply(lags, v)
    F = float(np.real(np.vdot(v, gv)))
    rhs = np.zeros((g.nx, g.ny), dtype=np.complex128)
    rhs[g.npml:g.nx - g.npml, g.j_src] = gv
    mu = ev.solver.solve(rhs)
    q = -2.0 * np.real(mu * z * _design_diag_weight(g))          # dF/d eps_c
    col = q[:, g.j_pillar0:g.j_pillar1].sum(axis=1)             # fill is uniform in the pillar rows
    return F, _to_widths(g, col, widths), z, mu


def bruteforce_grad(ev: Evaluation, widths: np.ndarray, theta, weight):
    """(F_bf, dF_bf/dwidths) by differentiating each angle's |w^dag u_q|^2."""
    g = ev.g
    z = np.conj(reciprocal_field(g, ev.solver, ev.w))            # A^{-1} conj(w)
    kss = _design_diag_weight(g)
    F = 0.0
    col = np.zeros(g.nx)
    for th, cq in zip(theta, weight):
        u = ev.solver.solve(planewave_source(g, th))
        a = np.vdot(ev.w, u)
        F += cq * abs(a) ** 2
        dA_u = -(z * kss * u)                                     # w^dag du per unit d eps_c
        col += (2.0 * cq * np.real(np.conj(a) * dA_u))[:, g.j_pillar0:g.j_pillar1].sum(axis=1)
    return float(F), _to_widths(g, col, widths)


def rule_lags(g: Grid, theta, weight) -> np.ndarray:
    """Toeplitz lags of W_N = sum_q c_q b0(theta_q) b0(theta_q)^dag for a rule that is
    symmetric in theta (imaginary parts cancel pairwise)."""
    D = np.arange(g.n_src) * g.h
    out = np.zeros(g.n_src)
    for th, cq in zip(theta, weight):
        out += cq * math.cos(th) * np.cos(g.k_sub * math.sin(th) * D)
    return out
