"""Pins for the oracle's reciprocal average (Eq. 7) and brute-force average (Eq. 6).

* the discrete identity behind Eq. 7 holds exactly for ANY angle rule, with the
  Toeplitz matrix built directly from the sources b0 (not from the closed form);
* the paper's central claim: the brute-force Gauss-Legendre average converges to the
  reciprocal value with the closed-form W as the rule is refined;
* the quadratic form three ways (direct, FFT circulant embedding, angular spectrum);
* limits (vanishing cone = one normal-incidence solve) and mirror symmetry;
* reciprocity of the Green's function; the virtual-focus propagator at zero height
  and against an on-grid focus in a taller domain."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.grid import Grid, rasterize_eps, planewave_source, virtual_focus_kernel
from oracle.light import W_lags, quadrature_rule
from oracle.reciprocal import Evaluation, qform_direct, qform_fft, qform_spectral
from oracle.solve import Solver


def _rng_rule(seed, n, c):
    rng = np.random.default_rng(seed)
    th = rng.uniform(-c, c, n)
    return th, rng.uniform(0.1, 1.0, n)


@pytest.mark.parametrize("kind", [W.OBJ_POINT, W.OBJ_PLANEWAVE, W.OBJ_VIRTUAL_FOCUS])
def test_discrete_identity_exact_for_any_rule(kind):
    wl = W.tiny(kind=kind)
    ev = Evaluation(wl, W.widths(wl.grid.n_cells, 11))
    g = ev.g
    th, wq = _rng_rule(1, 9, math.radians(40))
    f = ev.fom_per_angle(th)
    brute = float(np.dot(wq, f))
    _, v = ev.reciprocal()
    xs = g.x_src()
    # W_N[i, l] = sum_q wq b0_q[i] conj(b0_q[l]), straight from the sources
    B = np.stack([planewave_source(g, t)[g.npml:g.nx - g.npml, g.j_src] for t in th], 1)
    WN = (B * wq[None, :]) @ B.conj().T
    recip = float(np.real(np.vdot(v, WN @ v)))
    assert abs(brute - recip) < 1e-12 * abs(brute)


@pytest.mark.parametrize("maker", [lambda: W.tiny(kind=W.OBJ_POINT),
                                   lambda: W.small(kind=W.OBJ_PLANEWAVE)])
def test_bruteforce_converges_to_reciprocal(maker):
    wl = maker()
    ev = Evaluation(wl, W.widths(wl.grid.n_cells, 3))
    F, _ = ev.reciprocal()
    errs = []
    for n in (4, 8, 16, 64):
        Fb, _, _, _ = ev.bruteforce(n)
        errs.append(abs(Fb - F) / F)
    assert errs[-1] < 1e-11, errs
    assert errs[0] > errs[-1]


@pytest.mark.slow
def test_bruteforce_c1_at_201_angles():
    wl = W.c1_concentrator()
    ev = Evaluation(wl, W.widths(50, 0), refine=1)
    F, _ = ev.reciprocal()
    Fb, _, _, _ = ev.bruteforce(201)
    assert abs(Fb - F) / F < 1e-9


def test_qform_three_ways_and_positive():
    rng = np.random.default_rng(0)
    k_s = 2 * math.pi * math.sqrt(2.1)
    h = 0.05
    for n, light in ((1, W.Light(W.LIGHT_CONE, c=0.3)),
                     (37, W.Light(W.LIGHT_CONE, c=0.35)),
                     (300, W.Light(W.LIGHT_ANNULUS, th1=0.17, th2=0.52))):
        v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        lags = W_lags(light, k_s, h, n)
        d = qform_direct(v, lags)
        f = qform_fft(v, lags)
        th, wq = quadrature_rule(light, 400)
        s = qform_spectral(v, h * np.arange(n), k_s, th, wq)
        T = lags[np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])]
        dense = float(np.real(v.conj() @ T @ v))
        assert d > 0
        assert abs(d - dense) < 1e-12 * abs(dense)
        assert abs(d - f) < 1e-12 * abs(d)
        assert abs(d - s) < 1e-10 * abs(d)


def test_vanishing_cone_reduces_to_normal_incidence():
    wl = W.small(kind=W.OBJ_POINT)
    wl.light = W.Light(W.LIGHT_CONE, c=1e-4)
    ev = Evaluation(wl, W.widths(wl.grid.n_cells, 5))
    F, _ = ev.reciprocal()
    f0 = ev.fom_per_angle([0.0])[0]
    assert abs(F - f0) / f0 < 1e-6


def test_mirror_symmetry():
    wl = W.small(kind=W.OBJ_PLANEWAVE)
    wl.objective.theta_out = 0.0
    ws = W.widths(wl.grid.n_cells, 8)
    F1, v1 = Evaluation(wl, ws).reciprocal()
    F2, v2 = Evaluation(wl, ws[::-1].copy()).reciprocal()
    assert abs(F1 - F2) < 1e-12 * F1
    assert np.max(np.abs(v1 - v2[::-1])) < 1e-11 * np.max(np.abs(v1))


def test_green_reciprocity():
    wl = W.tiny()
    g = Grid(wl.grid)
    s = Solver(g, rasterize_eps(g, W.widths(3, 4)))
    a, b = (5, 7), (g.nx - 9, g.ny - 12)
    ea = np.zeros((g.nx, g.ny), complex); ea[a] = 1
    eb = np.zeros((g.nx, g.ny), complex); eb[b] = 1
    ua, ub = s.solve(ea), s.solve(eb)
    assert abs(ua[b] - ub[a]) < 1e-13 * abs(ua[b])


def test_virtual_focus_zero_height_is_lattice_delta():
    g = Grid(W.tiny().grid)
    m = np.arange(-6, 7)
    K = virtual_focus_kernel(g, m * g.h, 0)
    want = (m == 0).astype(float)
    assert np.max(np.abs(K - want)) < 1e-13
    # half-integer offsets: band-limited interpolation, K = sinc(pi Delta / h)
    Kh = virtual_focus_kernel(g, (m + 0.5) * g.h, 0)
    z = math.pi * (m + 0.5)
    assert np.max(np.abs(Kh - np.sin(z) / z)) < 1e-13


def test_virtual_focus_matches_on_grid_focus():
    # Field of a planewave source; compare u at a node D rows above the monitor row
    # with sum_i K(x_f - x_i) u(x_i, j_m) in the same (tall, homogeneous-air) domain.
    # Summed over every column the propagator reproduces the node value up to PML
    # reflections; the objective itself keeps only the interior columns, which drops
    # the field that reached the side PML (a ~0.3% effect at this aperture).
    d = W.GridDesc(n_cells=150, ny=200, npml=20, rows_sub=10, rows_pillar=12)
    g = Grid(d)
    eps = rasterize_eps(g, W.widths(150, 2))
    s = Solver(g, eps, refine=0)
    u = s.solve(planewave_source(g, math.radians(3)))
    jm = g.j_pillar1 + 5
    D = 60
    i_f = g.nx // 2
    got = u[i_f, jm + D]
    K_all = virtual_focus_kernel(g, g.x(i_f) - g.x(np.arange(g.nx)), D)
    assert abs(np.sum(K_all * u[:, jm]) - got) / abs(got) < 5e-4
    K = virtual_focus_kernel(g, g.x(i_f) - g.x_src(), D)
    pred = np.sum(K * u[g.npml:g.nx - g.npml, jm])
    assert abs(pred - got) / abs(got) < 1e-2
    # a downward (wrong-branch) propagator is far off
    K_bad = np.conj(K_all)
    assert abs(np.sum(K_bad * u[:, jm]) - got) / abs(got) > 0.1


@pytest.mark.parametrize("maker", [W.c3_precision, W.c4_gradient])
def test_virtual_focus_quadrature_converged_at_workload_heights(maker):
    # The propagator integral at the heights the workloads use (C3: 990 rows with offsets
    # up to 500 wavelengths; C4: 390 rows): doubling the panels and raising the order of
    # the composite rule changes K by less than 1e-12 of its largest value, so the rule
    # the library evaluates (256 panels x 32 points) sits on a converged integral.
    wl = maker()
    g = Grid(wl.grid)
    dl = wl.objective.x_f - g.x_src()
    sel = np.concatenate([dl[::max(1, dl.size // 300)], dl[[0, -1, dl.size // 2]]])
    K = virtual_focus_kernel(g, sel, wl.objective.d_rows)
    K_fine = virtual_focus_kernel(g, sel, wl.objective.d_rows, panels=512, order=48)
    assert np.max(np.abs(K - K_fine)) < 1e-12 * np.max(np.abs(K_fine))
    assert np.max(np.abs(dl)) > (400 if wl.objective.d_rows > 900 else 90)
