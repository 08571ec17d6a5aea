"""Pins for the oracle's angular statistics and quadrature (no GPU)."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

import workloads as W
from oracle.light import gauss_legendre, W_of_delta, W_lags, quadrature_rule, rho, sinc


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33, 64, 201, 500])
def test_gauss_legendre_matches_numpy(n):
    x, w = gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 1e-14
    assert np.max(np.abs(w - wr)) < 1e-13 * max(1.0, wr.max())


@pytest.mark.parametrize("n", [4, 10, 31])
def test_gauss_legendre_exact_on_polynomials(n):
    x, w = gauss_legendre(n)
    for k in range(0, 2 * n, 1):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13


def test_quadrature_rule_mass_and_support():
    cone = W.Light(W.LIGHT_CONE, c=math.radians(20))
    th, wq = quadrature_rule(cone, 201)
    assert abs(wq.sum() - 1.0) < 1e-14                 # unit total power
    assert np.all(np.abs(th) < cone.c)
    ann = W.Light(W.LIGHT_ANNULUS, th1=math.radians(10), th2=math.radians(30))
    th, wq = quadrature_rule(ann, 1000)
    assert abs(wq.sum() - 1.0) < 1e-14
    a = np.abs(th)
    assert np.all((a > ann.th1) & (a < ann.th2))
    assert np.allclose(np.sort(th), np.sort(-th))        # symmetric rule


@pytest.mark.parametrize("light", [W.Light(W.LIGHT_CONE, c=math.radians(20)),
                                   W.Light(W.LIGHT_CONE, c=math.radians(60)),
                                   W.Light(W.LIGHT_ANNULUS, th1=math.radians(10),
                                           th2=math.radians(30))])
def test_W_closed_form_against_adaptive_quadrature(light):
    # W(Delta) = int rho(theta) cos(theta) exp(i k sin(theta) Delta) d theta
    k = 2 * math.pi * math.sqrt(2.1)
    ivs = [(-light.c, light.c)] if light.kind == W.LIGHT_CONE else \
        [(-light.th2, -light.th1), (light.th1, light.th2)]
    dens = 1 / (2 * light.c) if light.kind == W.LIGHT_CONE else 1 / (2 * (light.th2 - light.th1))
    for delta in (0.0, 0.013, 0.37, 1.0, 4.05, 17.3):
        re = sum(scipy.integrate.quad(lambda t: dens * math.cos(t) * math.cos(k * math.sin(t) * delta),
                                      a, b, epsabs=1e-15, epsrel=1e-14, limit=400)[0]
                 for a, b in ivs)
        im = sum(scipy.integrate.quad(lambda t: dens * math.cos(t) * math.sin(k * math.sin(t) * delta),
                                      a, b, epsabs=1e-15, epsrel=1e-14, limit=400)[0]
                 for a, b in ivs)
        got = float(W_of_delta(light, k, delta))
        assert abs(got - re) < 1e-13, (delta, got, re)
        assert abs(im) < 1e-13                       # real and even


def test_W_cone_bessel_series():
    # For the cone, W(D) = (1/2c) int_{-c}^{c} cos(t) cos(z sin t) dt with z = k D.
    # Jacobi-Anger: cos(z sin t) = J0(z) + 2 sum_m J_{2m}(z) cos(2 m t); integrating
    # term by term gives an independent series for W.
    c = math.radians(35)
    k = 2 * math.pi
    light = W.Light(W.LIGHT_CONE, c=c)
    for D in (0.2, 1.3, 6.0):
        z = k * D
        tot = scipy.special.jv(0, z) * 2 * math.sin(c)
        for m in range(1, 80):
            n = 2 * m
            # int_{-c}^{c} cos t cos(n t) dt
            I = math.sin((n + 1) * c) / (n + 1) + math.sin((n - 1) * c) / (n - 1)
            tot += 2 * scipy.special.jv(n, z) * I
        assert abs(tot / (2 * c) - float(W_of_delta(light, k, D))) < 1e-13


def test_W_small_argument_branch_is_continuous():
    z = np.array([0.0, 5e-5, 9.99999e-5, 1.00001e-4, 2e-4, 1e-3])
    exact = np.array([1.0] + [math.sin(t) / t for t in z[1:]])
    assert np.max(np.abs(sinc(z) - exact)) < 1e-16 * 4


def test_W_lags_user_passthrough_and_shape():
    lags = np.linspace(1, 0, 7)
    got = W_lags(W.Light(W.LIGHT_USER_LAGS, lags=lags), 1.0, 0.05, 7)
    assert np.array_equal(got, lags)
    with pytest.raises(ValueError):
        W_lags(W.Light(W.LIGHT_USER_LAGS, lags=lags), 1.0, 0.05, 8)
    c = W.Light(W.LIGHT_CONE, c=0.3)
    assert np.allclose(W_lags(c, 3.0, 0.05, 5), W_of_delta(c, 3.0, 0.05 * np.arange(5)))
    assert rho(c, 0.1) == pytest.approx(1 / 0.6) and rho(c, 0.31) == 0.0


# ---- tabulated densities (piecewise linear in theta, even)
def _tab_W(theta, rho_tab, k_s, delta):
    from oracle.light import W_tabulated
    return W_tabulated(theta, rho_tab, k_s, delta)


def test_tabulated_constant_density_reproduces_the_cone_and_annulus_closed_forms():
    import workloads as W
    from oracle.light import W_of_delta
    k_s = 2 * math.pi * math.sqrt(2.1)
    delta = 0.05 * np.arange(0, 4000, 7)
    c = math.radians(20)
    got = _tab_W([0.0, c], [1 / (2 * c)] * 2, k_s, delta)
    want = W_of_delta(W.Light(W.LIGHT_CONE, c=c), k_s, delta)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    t1, t2 = math.radians(10), math.radians(30)
    got = _tab_W([t1, t2], [1 / (2 * (t2 - t1))] * 2, k_s, delta)
    want = W_of_delta(W.Light(W.LIGHT_ANNULUS, th1=t1, th2=t2), k_s, delta)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_tabulated_density_against_adaptive_quadrature():
    # a curved profile sampled at uneven nodes: the composite rule against scipy's adaptive
    # quadrature of the same piecewise-linear density, segment by segment
    import scipy.integrate as si
    k_s = 2 * math.pi * math.sqrt(2.1)
    theta = np.sort(np.concatenate([[0.0], np.random.default_rng(7).uniform(0.02, 0.6, 11), [0.62]]))
    rho_tab = np.cos(2.5 * theta) ** 2
    for d in (0.0, 0.37, 3.05, 41.2):
        got = _tab_W(theta, rho_tab, k_s, [d])[0]
        ref = 0.0
        for q in range(theta.size - 1):
            a, b = theta[q], theta[q + 1]
            f = lambda t: 2 * (rho_tab[q] + (rho_tab[q + 1] - rho_tab[q]) * (t - a) / (b - a)) \
                * math.cos(t) * math.cos(k_s * math.sin(t) * d)
            ref += si.quad(f, a, b, epsabs=1e-15, epsrel=1e-14, limit=500)[0]
        assert abs(got - ref) < 1e-12 * max(1.0, abs(ref)), (d, got, ref)


def test_tabulated_density_vanishing_width_limit():
    # a narrow triangle of unit area around theta0: W -> 2 cos(theta0) cos(k_s sin(theta0) D),
    # to second order in the width (about e^2 (k_s D)^2 / 12)
    k_s = 2 * math.pi * math.sqrt(2.1)
    t0, e = 0.3, 1e-6
    got = _tab_W([t0 - e, t0, t0 + e], [0.0, 1 / e, 0.0], k_s, [0.0, 1.3, 7.9])
    want = 2 * math.cos(t0) * np.cos(k_s * math.sin(t0) * np.array([0.0, 1.3, 7.9]))
    assert np.max(np.abs(got - want)) < 1e-8
