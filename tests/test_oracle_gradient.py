"""Pins for the oracle's width gradient (Sec. 4.1: adjoint of v^dag W v).

* the fill derivative against central differences of the raster itself (the fill is
  piecewise linear in each width, so the difference quotient is exact up to rounding
  when no edge crosses a column boundary);
* the adjoint gradient against central differences of F with a fresh factorisation
  per perturbed design, for every objective kind and both angular densities;
* the adjoint gradient with the Toeplitz lags of a quadrature rule against the
  gradient of the brute-force sum over that rule, differentiated angle by angle
  (the two agree exactly, since F_bf = v^dag W_N v for a symmetric rule);
* mirror symmetry of the gradient for a mirror-symmetric design and objective."""

import numpy as np
import pytest

import workloads as W
from oracle.grid import rasterize_eps
from oracle.gradient import (avg_intensity_grad, bruteforce_grad, fill_derivative,
                             rule_lags)
from oracle.light import quadrature_rule
from oracle.reciprocal import Evaluation


def _clear_widths(n, seed, h=0.05, margin=2e-3):
    """Seeded widths whose edges sit at least `margin` from every column boundary
    (pillar centres lie on boundaries, so the edge offset is (w/2) mod h)."""
    w = W.widths(n, seed)
    r = np.mod(w / 2, h)
    bad = (r < margin) | (r > h - margin)
    w[bad] += 4 * margin
    return w


def _F(wl, widths):
    ev = Evaluation(wl, widths)
    F, _ = ev.reciprocal()
    return F


def test_fill_derivative_matches_raster_differences():
    wl = W.small(n_cells=6)
    from oracle.grid import Grid
    g = Grid(wl.grid)
    w = _clear_widths(6, 3)
    D = fill_derivative(g, w)
    d = g.d
    jp = g.j_pillar0
    step = 1e-4
    for m in range(6):
        e = np.zeros(6)
        e[m] = step
        fd = (rasterize_eps(g, w + e)[:, jp] - rasterize_eps(g, w - e)[:, jp]) / (2 * step)
        np.testing.assert_allclose(fd, D[:, m] * (d.eps_pillar - d.eps_air), rtol=0, atol=1e-8)
        # exactly two edges per pillar: total fill rate 1/h
        assert D[:, m].sum() == pytest.approx(1.0 / g.h, rel=1e-15)


def test_fill_derivative_edges_straddle_the_centre():
    # pillar centres lie on column boundaries, so the two edges always fall in two
    # different columns, each with rate 1/(2h), even for a pillar narrower than h
    wl = W.small(n_cells=2)
    from oracle.grid import Grid
    g = Grid(wl.grid)
    w = np.array([0.03, 0.2])
    D = fill_derivative(g, w)
    assert np.count_nonzero(D[:, 0]) == 2
    w = np.array([0.2, 0.2])
    D = fill_derivative(g, w)
    assert np.count_nonzero(D[:, 0]) == 2 and np.all(D[D != 0] == 0.5 / g.h)


@pytest.mark.parametrize("kind", [W.OBJ_POINT, W.OBJ_PLANEWAVE, W.OBJ_VIRTUAL_FOCUS])
@pytest.mark.parametrize("light", ["cone", "annulus"])
def test_adjoint_gradient_matches_central_differences(kind, light):
    wl = W.tiny(kind=kind, n_cells=4)
    if light == "annulus":
        wl.light = W.Light(W.LIGHT_ANNULUS, th1=W.deg(5), th2=W.deg(25))
    w = _clear_widths(4, 7)
    ev = Evaluation(wl, w)
    F, grad, _, _ = avg_intensity_grad(ev, w)
    F_ref, _ = ev.reciprocal()
    assert F == pytest.approx(F_ref, rel=1e-12)
    step = 1e-6
    fd = np.empty(4)
    for m in range(4):
        e = np.zeros(4)
        e[m] = step
        fd[m] = (_F(wl, w + e) - _F(wl, w - e)) / (2 * step)
    scale = np.max(np.abs(grad))
    assert scale > 0
    np.testing.assert_allclose(grad, fd, rtol=0, atol=1e-8 * scale)


def test_adjoint_matches_bruteforce_gradient_on_same_rule():
    wl = W.small(n_cells=5, ny=56)
    w = _clear_widths(5, 9)
    ev = Evaluation(wl, w)
    theta, wq = quadrature_rule(wl.light, 16)
    F_bf, g_bf = bruteforce_grad(ev, w, theta, wq)
    F_adj, g_adj, _, _ = avg_intensity_grad(ev, w, lags=rule_lags(ev.g, theta, wq))
    assert F_adj == pytest.approx(F_bf, rel=1e-11)
    np.testing.assert_allclose(g_adj, g_bf, rtol=0, atol=1e-10 * np.max(np.abs(g_bf)))


@pytest.mark.parametrize("kind", [W.OBJ_PLANEWAVE, W.OBJ_VIRTUAL_FOCUS])
def test_gradient_mirror_symmetry(kind):
    wl = W.small(n_cells=6, kind=kind)
    if kind == W.OBJ_PLANEWAVE:
        wl.objective.theta_out = 0.0
    half = _clear_widths(3, 21)
    w = np.concatenate([half, half[::-1]])
    ev = Evaluation(wl, w)
    _, grad, _, _ = avg_intensity_grad(ev, w)
    np.testing.assert_allclose(grad, grad[::-1], rtol=0, atol=1e-9 * np.max(np.abs(grad)))


def test_gradient_is_a_descent_direction():
    # one small step along the gradient raises F by about |grad|^2 * step
    wl = W.tiny(kind=W.OBJ_PLANEWAVE, n_cells=4)
    w = _clear_widths(4, 2)
    ev = Evaluation(wl, w)
    F0, grad, _, _ = avg_intensity_grad(ev, w)
    t = 1e-7 / np.max(np.abs(grad))
    F1 = _F(wl, w + t * grad)
    assert F1 - F0 == pytest.approx(t * np.dot(grad, grad), rel=1e-3)
