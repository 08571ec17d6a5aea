"""Incoherent light statistics and quadrature (oracle; test infrastructure only).

Angular density rho(theta) = <|a(theta)|^2>, normalised to unit total power
(Sec. 3: <|a|^2> = 1/2c on the cone [-c, c]).  Angles are measured in the medium of
the source plane (the substrate, index n_s = sqrt(eps_sub)), as k_x = n (2 pi/lambda)
sin(theta) in Eq. 3.

Cross-correlation of the equivalent currents (Eq. 3 with uncorrelated angles, Sec. 3):
with the unit-power amplitude sqrt(cos theta) of b0(theta),

    W(Delta) = int rho(theta) cos(theta) exp(i k_s sin(theta) Delta) d theta .

This is the exact reading of Eq. 4 and of the annulus formula of Sec. 5.1: the
cos(theta) Jacobian turns the uniform-in-theta density into a uniform density in
sin(theta), so

    cone    W = (sin c / c) sinc(k_s Delta sin c)
    annulus W = [sin th2 sinc(k_s Delta sin th2) - sin th1 sinc(k_s Delta sin th1)] / (th2 - th1)

with sinc(z) = sin(z)/z.  (The printed formulas drop the Jacobian and the index and
carry theta where sin(theta) is exact; the printed forms are still reachable through
LIGHT_USER_LAGS.)  W is real and even for these symmetric densities.

A tabulated density (LIGHT_TABULATED) is given at nodes 0 <= theta_0 < ... < theta_{n-1}
< pi/2, linear in theta between nodes, zero outside, and even (rho(-theta) = rho(theta)), so

    W(Delta) = 2 int_{theta_0}^{theta_{n-1}} rho(theta) cos(theta) cos(k_s sin(theta) Delta) d theta,

integrated here segment by segment with a composite Gauss-Legendre rule in theta.
"""
from __future__ import annotations

import math

import numpy as np

from workloads import Light, LIGHT_CONE, LIGHT_ANNULUS, LIGHT_USER_LAGS, LIGHT_TABULATED


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (Sec. 5.2).  Roots of P_n by Newton's
    method on the three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},
    started at cos(pi (k - 1/4) / (n + 1/2)); weights 2 / ((1 - x^2) P_n'(x)^2)."""
    if n < 1:
        raise ValueError("n >= 1")
    k = np.arange(1, n + 1)
    x = np.cos(math.pi * (k - 0.25) / (n + 0.5))
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for m in range(1, n):
            p0, p1 = p1, ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
        # p1 = P_n, p0 = P_{n-1};  P_n' = n (x P_n - P_{n-1}) / (x^2 - 1)
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0 = np.ones_like(x)
    p1 = x.copy()
    for m in range(1, n):
        p0, p1 = p1, ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
    dp = n * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def rho(light: Light, theta):
    """Angular density (unit total mass)."""
    theta = np.asarray(theta, dtype=np.float64)
    if light.kind == LIGHT_CONE:
        return np.where(np.abs(theta) <= light.c, 1.0 / (2.0 * light.c), 0.0)
    if light.kind == LIGHT_ANNULUS:
        a = np.abs(theta)
        inside = (a >= light.th1) & (a <= light.th2)
        return np.where(inside, 1.0 / (2.0 * (light.th2 - light.th1)), 0.0)
    raise ValueError("rho is defined for cone and annulus light")


def intervals(light: Light):
    if light.kind == LIGHT_CONE:
        return [(-light.c, light.c)]
    if light.kind == LIGHT_ANNULUS:
        return [(-light.th2, -light.th1), (light.th1, light.th2)]
    raise ValueError("no angular support for user lags")


def quadrature_rule(light: Light, n: int):
    """Brute-force rule {theta_q, Omega_q rho(theta_q)} (Sec. 5.2): n Gauss-Legendre
    points on the cone, or n/2 on each interval of the annulus."""
    ivs = intervals(light)
    per = n // len(ivs)
    if per < 1 or per * len(ivs) != n:
        raise ValueError("annulus rules need an even number of points")
    th, wt = [], []
    x, w = gauss_legendre(per)
    for a, b in ivs:
        th.append(0.5 * (b - a) * x + 0.5 * (a + b))
        wt.append(0.5 * (b - a) * w)
    th = np.concatenate(th)
    wt = np.concatenate(wt)
    return th, wt * rho(light, th)


def sinc(z):
    z = np.asarray(z, dtype=np.float64)
    out = np.ones_like(z)
    big = np.abs(z) > 1e-4
    out[big] = np.sin(z[big]) / z[big]
    zs = z[~big]
    out[~big] = 1.0 - zs * zs / 6.0 + zs ** 4 / 120.0
    return out


def W_of_delta(light: Light, k_s: float, delta):
    """Closed-form W(Delta) (module docstring)."""
    delta = np.asarray(delta, dtype=np.float64)
    if light.kind == LIGHT_CONE:
        c = light.c
        return (math.sin(c) / c) * sinc(k_s * delta * math.sin(c))
    if light.kind == LIGHT_ANNULUS:
        s1, s2 = math.sin(light.th1), math.sin(light.th2)
        return (s2 * sinc(k_s * delta * s2) - s1 * sinc(k_s * delta * s1)) / (light.th2 - light.th1)
    raise ValueError("closed form only for cone and annulus")


def W_tabulated(theta, rho_tab, k_s: float, delta, order: int = 20) -> np.ndarray:
    """W(Delta) of a tabulated, piecewise-linear, even density (module docstring): on each
    segment, sub-panels in theta no wider than a third of the shortest oscillation period
    of cos(k_s sin(theta) Delta) over the requested Delta, `order` Gauss-Legendre points each."""
    theta = np.asarray(theta, dtype=np.float64)
    rho_tab = np.asarray(rho_tab, dtype=np.float64)
    delta = np.atleast_1d(np.asarray(delta, dtype=np.float64))
    dmax = float(np.max(np.abs(delta))) if delta.size else 0.0
    x, w = gauss_legendre(order)
    th_all, c_all = [], []
    for q in range(theta.size - 1):
        a, b = theta[q], theta[q + 1]
        # |d/dtheta (k_s sin(theta) Delta)| <= k_s Delta: period >= 2 pi / (k_s Delta)
        panels = max(1, int(math.ceil((b - a) * k_s * dmax / (2 * math.pi / 3))))
        edges = np.linspace(a, b, panels + 1)
        mid = 0.5 * (edges[1:] + edges[:-1])
        half = 0.5 * (edges[1:] - edges[:-1])
        th = (mid[:, None] + half[:, None] * x[None, :]).ravel()
        wt = (half[:, None] * w[None, :]).ravel()
        r = rho_tab[q] + (rho_tab[q + 1] - rho_tab[q]) * (th - a) / (b - a)
        th_all.append(th)
        c_all.append(2.0 * wt * r * np.cos(th))
    th = np.concatenate(th_all)
    cw = np.concatenate(c_all)
    s = np.sin(th)
    out = np.empty(delta.shape)
    for i0 in range(0, delta.size, 512):
        d = delta[i0:i0 + 512]
        out[i0:i0 + 512] = np.cos(k_s * np.outer(d, s)) @ cw
    return out


def W_lags(light: Light, k_s: float, h: float, n: int) -> np.ndarray:
    """W(m h) for m = 0..n-1 (the Toeplitz symbol on the source plane)."""
    if light.kind == LIGHT_TABULATED:
        return W_tabulated(light.theta, light.rho, k_s, h * np.arange(n))
    if light.kind == LIGHT_USER_LAGS:
        lags = np.asarray(light.lags, dtype=np.float64)
        if lags.shape != (n,):
            raise ValueError("user lags need n_src entries")
        return lags.copy()
    return W_of_delta(light, k_s, h * np.arange(n))
