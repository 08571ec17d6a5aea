"""Correlated incoherent light and multi-output objectives (oracle; test infrastructure only).

Correlated angles (Eq. 5, Eq. 3).  With the angular amplitude correlation
<a(theta) a*(theta')> given on a quadrature rule (theta_q, Omega_q) as a Hermitian matrix
C[q, q'], the equivalent currents b = sum_q Omega_q a_q b0(theta_q) have the
cross-correlation

    W = <b b^dag> = sum_{q,q'} Omega_q Omega_q' C[q, q'] b0(theta_q) b0(theta_q')^dag ,

a general (not Toeplitz) Hermitian matrix on the source plane, and Eq. 7 gives
F = v^dag W v with the same single reciprocal solve.  The forward form of Eq. 5 on the
same rule is sum_{q,q'} Omega_q Omega_q' C[q, q'] (w^dag u_q) conj(w^dag u_q'), one forward
solve per angle.  Uncorrelated light is C = diag(rho_q / Omega_q).

Multi-output objectives (Sec. 6: averages over several spots or modes): each output o has
its own w_o and F_o = v_o^dag W v_o with v_o = A^{-dag} w_o; the trace objective is their sum.
"""
from __future__ import annotations

import numpy as np

from oracle.grid import Grid, objective_vector, planewave_source
from oracle.reciprocal import Evaluation, reciprocal_field, source_plane


def angular_sources(g: Grid, theta) -> np.ndarray:
    """B[:, q] = b0(theta_q) on the source plane (n_src x nq)."""
    xs = g.x_src()
    th = np.asarray(theta, dtype=np.float64)
    return np.sqrt(np.cos(th))[None, :] * np.exp(1j * g.k_sub * np.sin(th)[None, :] * xs[:, None])


def correlated_W(g: Grid, theta, weight, C) -> np.ndarray:
    """Dense W of Eq. 3 for the quadrature (theta, weight) and correlation matrix C."""
    B = angular_sources(g, theta)
    Om = np.asarray(weight, dtype=np.float64)
    M = Om[:, None] * np.asarray(C, dtype=np.complex128) * Om[None, :]
    return B @ M @ B.conj().T


def qform_dense(v: np.ndarray, W: np.ndarray) -> float:
    """Re(v^dag W v) for a Hermitian W."""
    return float(np.real(np.vdot(v, W @ v)))


def avg_intensity_correlated(ev: Evaluation, theta, weight, C) -> float:
    """Reciprocal value v^dag W v with the W of Eq. 3 (one reciprocal solve)."""
    v = source_plane(ev.g, reciprocal_field(ev.g, ev.solver, ev.w))
    return qform_dense(v, correlated_W(ev.g, theta, weight, C))


def forward_correlated(ev: Evaluation, theta, weight, C) -> float:
    """Eq. 5 on the rule: sum_{q,q'} Om_q Om_q' C[q,q'] (w^dag u_q) conj(w^dag u_q')."""
    g = ev.g
    alpha = np.array([np.vdot(ev.w, ev.solver.solve(planewave_source(g, t))) for t in theta])
    Om = np.asarray(weight, dtype=np.float64)
    M = Om[:, None] * np.asarray(C, dtype=np.complex128) * Om[None, :]
    return float(np.real(alpha @ M @ alpha.conj()))


def coherent_superposition(ev: Evaluation, theta, weight, a) -> float:
    """|w^dag A^{-1} b|^2 for the single source b = sum_q Omega_q a_q b0(theta_q): the fully
    coherent light whose correlation is C = a a^dag."""
    g = ev.g
    b = np.zeros((g.nx, g.ny), dtype=np.complex128)
    for t, om, aq in zip(theta, weight, a):
        b += om * aq * planewave_source(g, t)
    return float(abs(np.vdot(ev.w, ev.solver.solve(b))) ** 2)


def avg_intensity_multi(ev: Evaluation, objectives, lags) -> np.ndarray:
    """F_o = v_o^dag W v_o for each objective (Toeplitz W from lags), one solve each."""
    from oracle.reciprocal import qform_direct
    out = []
    for o in objectives:
        w = objective_vector(ev.g, o)
        v = source_plane(ev.g, reciprocal_field(ev.g, ev.solver, w))
        out.append(qform_direct(v, lags))
    return np.array(out)
