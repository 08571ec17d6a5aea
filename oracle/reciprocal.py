"""Reciprocal and brute-force averaged figure of merit (oracle; test infrastructure only).

Reciprocal (Eq. 7, Sec. 4.1):  <|w^dag u|^2> = v^dag W v  with  v = A^{-dag} w.
A is complex symmetric (A = A^T), so A^{-dag} w = conj(A^{-1} conj(w)): one
factorisation serves both directions.  Only the values of v on the source plane
(row j_src, interior columns S) enter, since b is supported there:

    F_rec = sum_{i,l in S} conj(v_i) W(x_i - x_l) v_l .

Brute force (Eq. 6, Sec. 5.2):  F_bf = sum_q Omega_q rho(theta_q) |w^dag A^{-1} b0(theta_q)|^2
over a Gauss-Legendre rule on the angular support.

Sums over the source plane carry no h factors (arbitrary units, Sec. 5.1).
"""
from __future__ import annotations

import math
import time

import numpy as np

from workloads import Workload
from oracle.grid import Grid, rasterize_eps, objective_vector, planewave_source
from oracle.light import W_lags, quadrature_rule
from oracle.solve import Solver


def reciprocal_field(g: Grid, solver: Solver, w: np.ndarray) -> np.ndarray:
    """v = A^{-dag} w on the whole grid (nx, ny)."""
    z = solver.solve(np.conj(w))
    return np.conj(z)


def source_plane(g: Grid, field: np.ndarray) -> np.ndarray:
    return field[g.npml:g.nx - g.npml, g.j_src].copy()


def qform_direct(v: np.ndarray, lags: np.ndarray, block: int = 2048) -> float:
    """sum_{i,l} conj(v_i) W_{|i-l|} v_l by rows of the Toeplitz matrix, in blocks."""
    n = v.size
    total = 0.0
    idx = np.arange(n)
    for s in range(0, n, block):
        rows = idx[s:s + block]
        T = lags[np.abs(rows[:, None] - idx[None, :])]
        total += float(np.real(np.vdot(v[s:s + block], T @ v)))
    return total


def qform_fft(v: np.ndarray, lags: np.ndarray) -> float:
    """Same form through a circulant embedding of the Toeplitz matrix (Sec. 4.1: the
    convolution of W with the reciprocal field, evaluated with FFTs)."""
    n = v.size
    L = 1 << int(math.ceil(math.log2(2 * n)))
    col = np.zeros(L)
    col[:n] = lags
    col[L - n + 1:] = lags[1:][::-1]
    vv = np.zeros(L, dtype=np.complex128)
    vv[:n] = v
    Tv = np.fft.ifft(np.fft.fft(col) * np.fft.fft(vv))[:n]
    return float(np.real(np.vdot(v, Tv)))


def qform_spectral(v: np.ndarray, xs: np.ndarray, k_s: float, theta, weight) -> float:
    """int rho(theta) cos(theta) |sum_l v_l exp(-i k_s sin(theta) x_l)|^2 d theta with a
    quadrature rule (theta, weight = Omega * rho): the angular-spectrum form of v^dag W v."""
    tot = 0.0
    for th, wq in zip(theta, weight):
        a = np.sum(v * np.exp(-1j * k_s * math.sin(th) * xs))
        tot += wq * math.cos(th) * abs(a) ** 2
    return float(tot)


class Evaluation:
    """One design of one workload: assembled, factored, ready to evaluate."""

    def __init__(self, wl: Workload, widths: np.ndarray, refine: int = 2):
        self.wl = wl
        self.g = Grid(wl.grid)
        self.eps = rasterize_eps(self.g, widths)
        self.solver = Solver(self.g, self.eps, refine=refine)
        self.w = objective_vector(self.g, wl.objective)

    def lags(self) -> np.ndarray:
        return W_lags(self.wl.light, self.g.k_sub, self.g.h, self.g.n_src)

    def reciprocal(self):
        """(F_rec, v on the source plane)."""
        v_full = reciprocal_field(self.g, self.solver, self.w)
        v = source_plane(self.g, v_full)
        return qform_direct(v, self.lags()), v

    def fom_per_angle(self, theta) -> np.ndarray:
        """|w^dag u(theta)|^2 for each angle (forward solves)."""
        g = self.g
        B = np.stack([planewave_source(g, t) for t in theta], axis=-1)
        U = self.solver.solve(B)
        amp = np.einsum("ij,ijq->q", np.conj(self.w), U)
        return np.abs(amp) ** 2

    def bruteforce(self, n: int):
        """(F_bf, theta, Omega*rho, per-angle FOM) with an n-point rule."""
        theta, wq = quadrature_rule(self.wl.light, n)
        f = self.fom_per_angle(theta)
        return float(np.dot(wq, f)), theta, wq, f


def timed_reciprocal(wl: Workload, widths: np.ndarray, refine: int = 2):
    """(F_rec, seconds) for one cold evaluation: raster, assemble, factor, solve, form."""
    t0 = time.perf_counter()
    ev = Evaluation(wl, widths, refine=refine)
    F, _ = ev.reciprocal()
    return F, time.perf_counter() - t0
