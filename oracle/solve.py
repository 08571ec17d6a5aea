"""Linear solves with A (oracle; test infrastructure only).

u = A^{-1} b (Sec. 4.1).  The factorisation step is a library sparse LU
(SuperLU through scipy); the residual of each refinement step is evaluated by the
stencil in double-double arithmetic (Knuth's TwoSum, Dekker's TwoProduct with
Veltkamp splitting), so the refined solution carries a forward error near the
FP64 unit roundoff rather than condition-number times it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from oracle.grid import Grid, assemble, stencil_coefficients


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _split(a):
    c = 134217729.0 * a            # 2^27 + 1
    hi = c - (c - a)
    return hi, a - hi


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


class _DD:
    """Accumulator s + e for real arrays."""

    def __init__(self, x):
        self.s = np.array(x, dtype=np.float64, copy=True)
        self.e = np.zeros_like(self.s)

    def add(self, x):
        self.s, err = _two_sum(self.s, x)
        self.e += err

    def add_prod(self, a, b, sign=1.0):
        p, err = _two_prod(a, b)
        self.add(sign * p)
        self.e += sign * err

    def value(self):
        return self.s + self.e


def residual_dd(coeffs, b: np.ndarray, u: np.ndarray) -> np.ndarray:
    """r = b - A u on the (nx, ny) grid, accumulated in double-double."""
    diag, cxp, cyp = coeffs
    rr = _DD(b.real)
    ri = _DD(b.imag)

    def sub_prod(region, c, x):
        # (cr + i ci)(xr + i xi) subtracted from r[region]
        cr, ci, xr, xi = c.real, c.imag, x.real, x.imag
        for acc, terms in ((rr, ((cr, xr, -1.0), (ci, xi, +1.0))),
                           (ri, ((cr, xi, -1.0), (ci, xr, -1.0)))):
            sub = _DD(acc.s[region])
            sub.e = acc.e[region].copy()
            for a_, b_, sg in terms:
                sub.add_prod(a_, b_, sg)
            acc.s[region] = sub.s
            acc.e[region] = sub.e

    full = (slice(None), slice(None))
    sub_prod(full, diag, u)
    sub_prod((slice(0, -1), slice(None)), cxp, u[1:])
    sub_prod((slice(1, None), slice(None)), cxp, u[:-1])
    sub_prod((slice(None), slice(0, -1)), cyp, u[:, 1:])
    sub_prod((slice(None), slice(1, None)), cyp, u[:, :-1])
    return rr.value() + 1j * ri.value()


class Solver:
    """LU of A for one design; solve() refines every right-hand side."""

    def __init__(self, g: Grid, eps: np.ndarray, refine: int = 2):
        self.g = g
        self.coeffs = stencil_coefficients(g, eps)
        self.A = assemble(g, eps)
        self.lu = spla.splu(self.A)
        self.refine = refine

    def solve(self, b: np.ndarray) -> np.ndarray:
        """b: (nx, ny) or (nx, ny, nrhs); returns u of the same shape."""
        g = self.g
        multi = b.ndim == 3
        B = b.reshape(g.N, -1)
        U = self.lu.solve(np.ascontiguousarray(B))
        U = U.reshape(B.shape)
        for _ in range(self.refine):
            R = np.empty_like(U)
            for c in range(U.shape[1]):
                R[:, c] = residual_dd(self.coeffs, B[:, c].reshape(g.nx, g.ny),
                                      U[:, c].reshape(g.nx, g.ny)).ravel()
            U = U + self.lu.solve(R).reshape(U.shape)
        return U.reshape(b.shape) if multi else U.reshape(g.nx, g.ny)

    def solve_plain(self, b: np.ndarray) -> np.ndarray:
        """Unrefined LU solve (for timing and for the multi-angle brute force)."""
        g = self.g
        B = b.reshape(g.N, -1)
        return self.lu.solve(np.ascontiguousarray(B)).reshape(b.shape)
