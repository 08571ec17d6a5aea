"""Pins for the oracle's correlated-light and multi-output forms.

* the reciprocal value v^dag W v with the W of Eq. 3 equals the forward double sum of
  Eq. 5 (one forward solve per angle) for a random Hermitian correlation, every objective;
* a rank-one correlation C = a a^dag is fully coherent light: it equals one forward
  solve with the superposed source (pins the conjugation orientation of Eq. 5);
* a diagonal correlation reproduces the uncorrelated brute force of Eq. 6, and its dense
  W equals the Toeplitz W of the same rule;
* the multi-output values equal one reciprocal evaluation per objective."""
import numpy as np
import pytest

import workloads as W
from oracle.correlated import (avg_intensity_correlated, avg_intensity_multi, coherent_superposition,
                               correlated_W, forward_correlated, qform_dense)
from oracle.gradient import rule_lags
from oracle.light import quadrature_rule
from oracle.reciprocal import Evaluation, qform_direct, reciprocal_field, source_plane


def _rule(seed, n, c):
    rng = np.random.default_rng(seed)
    return np.sort(rng.uniform(-c, c, n)), rng.uniform(0.05, 0.2, n)


def _hermitian_psd(seed, n):
    rng = np.random.default_rng(seed)
    G = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return G @ G.conj().T / n


@pytest.mark.parametrize("kind", [W.OBJ_POINT, W.OBJ_PLANEWAVE, W.OBJ_VIRTUAL_FOCUS])
def test_reciprocal_equals_forward_for_correlated_light(kind):
    wl = W.tiny(kind=kind, n_cells=4)
    ev = Evaluation(wl, W.widths(4, 3))
    theta, om = _rule(1, 7, 0.6)
    C = _hermitian_psd(2, 7)
    F_rec = avg_intensity_correlated(ev, theta, om, C)
    F_fwd = forward_correlated(ev, theta, om, C)
    assert F_rec > 0
    assert F_rec == pytest.approx(F_fwd, rel=1e-11)


def test_rank_one_correlation_is_one_coherent_solve():
    wl = W.tiny(kind=W.OBJ_PLANEWAVE, n_cells=4)
    ev = Evaluation(wl, W.widths(4, 5))
    theta, om = _rule(3, 6, 0.5)
    rng = np.random.default_rng(4)
    a = rng.normal(size=6) + 1j * rng.normal(size=6)
    C = np.outer(a, a.conj())
    assert avg_intensity_correlated(ev, theta, om, C) == pytest.approx(
        coherent_superposition(ev, theta, om, a), rel=1e-11)
    # conjugating the correlation (the other orientation of Eq. 5) gives a different value
    assert abs(avg_intensity_correlated(ev, theta, om, C.conj())
               - coherent_superposition(ev, theta, om, a)) > 1e-3 * coherent_superposition(ev, theta, om, a)


def test_diagonal_correlation_is_the_uncorrelated_brute_force():
    wl = W.small(kind=W.OBJ_VIRTUAL_FOCUS)
    ev = Evaluation(wl, W.widths(wl.grid.n_cells, 6))
    theta, wq = quadrature_rule(wl.light, 12)            # wq = Omega_q rho_q
    F_bf, _, _, _ = ev.bruteforce(12)
    # Omega = sqrt(wq), C = identity  ->  Omega C Omega = diag(wq)
    F_c = avg_intensity_correlated(ev, theta, np.sqrt(wq), np.eye(12))
    assert F_c == pytest.approx(F_bf, rel=1e-11)
    # and its dense W is the Toeplitz W of the rule
    v = source_plane(ev.g, reciprocal_field(ev.g, ev.solver, ev.w))
    Wd = correlated_W(ev.g, theta, np.sqrt(wq), np.eye(12))
    assert np.allclose(Wd, Wd.conj().T, rtol=0, atol=1e-15 * np.abs(Wd).max())
    assert qform_dense(v, Wd) == pytest.approx(qform_direct(v, rule_lags(ev.g, theta, wq)), rel=1e-12)


def test_correlated_value_is_linear_in_the_correlation():
    wl = W.tiny(kind=W.OBJ_POINT, n_cells=3)
    ev = Evaluation(wl, W.widths(3, 8))
    theta, om = _rule(5, 5, 0.7)
    C1, C2 = _hermitian_psd(6, 5), _hermitian_psd(7, 5)
    f = lambda C: avg_intensity_correlated(ev, theta, om, C)
    assert f(2.0 * C1 + 0.5 * C2) == pytest.approx(2.0 * f(C1) + 0.5 * f(C2), rel=1e-12)


def test_multi_output_values_equal_single_evaluations():
    wl = W.small(kind=W.OBJ_PLANEWAVE)
    ws = W.widths(wl.grid.n_cells, 9)
    objs = [W.Objective(kind=W.OBJ_PLANEWAVE, monitor_row=wl.objective.monitor_row, theta_out=t)
            for t in (0.0, 0.05, -0.1)]
    ev = Evaluation(wl, ws)
    Fm = avg_intensity_multi(ev, objs, ev.lags())
    for o, F in zip(objs, Fm):
        wl_o = W.Workload("o", wl.grid, o, wl.light, 0)
        assert F == pytest.approx(Evaluation(wl_o, ws).reciprocal()[0], rel=1e-13)
