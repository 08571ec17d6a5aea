"""Pins for the oracle's grid, permittivity and operator (no GPU).

Each test checks the oracle against something other than itself: a hand-derived
fill fraction, exact symmetry, the continuum Green's function (i/4) H0^(1)(k r),
the discrete Green identity (flux conservation), the lattice dispersion relation
of a planewave, and a dense LAPACK solve."""
import math

import numpy as np
import pytest
import scipy.special

import workloads as W
from oracle.grid import (Grid, rasterize_eps, assemble, stencil_coefficients, apply_A,
                         planewave_source)
from oracle.solve import Solver, residual_dd


def test_sizes_of_the_stated_workloads():
    # nx = 20 px/lambda * width + 2 PML; the stated grids are 440, 4040, 20040 wide.
    for fn, nx, ny in ((W.c1_concentrator, 440, 128), (W.c2_collimator, 4040, 160),
                       (W.c3_precision, 20040, 224)):
        g = Grid(fn().grid)
        assert (g.nx, g.ny) == (nx, ny)
        assert g.n_src == nx - 40
        assert g.j_pillar1 - g.j_pillar0 == 12          # 0.6 lambda pillars


def test_raster_hand_values():
    # two cells of 8 columns (h = 0.05, p = 0.4); pillars [0.135, 0.265] and
    # [0.435, 0.765]: edge columns are covered 0.015/0.05 = 0.3.
    d = W.GridDesc(n_cells=2, ny=40, npml=4, rows_sub=4, rows_pillar=4)
    g = Grid(d)
    eps = rasterize_eps(g, np.array([0.13, 0.33]))
    f = (eps[4:-4, g.j_pillar0] - d.eps_air) / (d.eps_pillar - d.eps_air)
    want = [0, 0, .3, 1, 1, .3, 0, 0, .3, 1, 1, 1, 1, 1, 1, .3]
    assert np.allclose(f, want, atol=1e-12)
    assert np.all(eps[:, : g.j_pillar0] == d.eps_sub)
    assert np.all(eps[:, g.j_pillar1:] == d.eps_air)
    assert np.all(eps[:4, g.j_pillar0] == d.eps_air)     # no pillar in the x-PML


def test_raster_conserves_pillar_area():
    d = W.c1_concentrator().grid
    g = Grid(d)
    ws = W.widths(d.n_cells, 7)
    eps = rasterize_eps(g, ws)
    f = (eps[:, g.j_pillar0] - d.eps_air) / (d.eps_pillar - d.eps_air)
    assert abs(f.sum() * g.h - ws.sum()) < 1e-12
    assert f.min() >= 0 and f.max() <= 1 + 1e-13


def test_operator_is_complex_symmetric():
    wl = W.tiny()
    g = Grid(wl.grid)
    A = assemble(g, rasterize_eps(g, W.widths(3, 1)))
    assert (A - A.T).count_nonzero() == 0
    assert np.iscomplexobj(A.data)


def test_dense_solve_matches_lapack():
    wl = W.tiny()
    g = Grid(wl.grid)
    eps = rasterize_eps(g, W.widths(3, 2))
    A = assemble(g, eps).toarray()
    rng = np.random.default_rng(3)
    b = rng.standard_normal((g.nx, g.ny)) + 1j * rng.standard_normal((g.nx, g.ny))
    u_ref = np.linalg.solve(A, b.ravel()).reshape(g.nx, g.ny)
    u = Solver(g, eps).solve(b)
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-12
    # the stencil form of A agrees with the sparse matrix
    coeffs = stencil_coefficients(g, eps)
    assert np.allclose(apply_A(g, coeffs, u_ref), (A @ u_ref.ravel()).reshape(g.nx, g.ny),
                       rtol=0, atol=1e-9 * np.abs(b).max())


def test_double_double_residual_is_exact_to_rounding():
    from fractions import Fraction
    wl = W.tiny(n_cells=1, ny=24)
    d = wl.grid
    d.npml, d.rows_sub, d.rows_pillar = 4, 4, 4
    g = Grid(d)
    eps = rasterize_eps(g, np.array([0.2]))
    coeffs = stencil_coefficients(g, eps)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((g.nx, g.ny)) + 1j * rng.standard_normal((g.nx, g.ny))
    b = apply_A(g, coeffs, u) + 1e-9 * (rng.standard_normal(u.shape) + 0j)
    r = residual_dd(coeffs, b, u)
    A = assemble(g, eps).tocsr()
    F = Fraction
    worst = 0.0
    for k in range(g.N):
        i, j = divmod(k, g.ny)
        sr, si = F(b[i, j].real), F(b[i, j].imag)
        for p in range(A.indptr[k], A.indptr[k + 1]):
            a = A.data[p]
            x = u.ravel()[A.indices[p]]
            sr -= F(a.real) * F(x.real) - F(a.imag) * F(x.imag)
            si -= F(a.real) * F(x.imag) + F(a.imag) * F(x.real)
        worst = max(worst, abs(float(sr) - r[i, j].real), abs(float(si) - r[i, j].imag))
    # exact residual is ~1e-9; double-double keeps it to ~1e-25 absolute here
    assert worst < 1e-20


def _vacuum_desc(ppl, half_width_lambda=4):
    cell_px = ppl * 2 // 5                 # p = 0.4 lambda
    n_cells = int(2 * half_width_lambda / 0.4)
    ny = 2 * half_width_lambda * ppl + 2 * ppl
    return W.GridDesc(n_cells=n_cells, ny=ny, ppl=ppl, cell_px=cell_px, npml=ppl,
                      rows_sub=ppl, rows_pillar=ppl // 2, eps_pillar=1.0, eps_sub=1.0,
                      eps_air=1.0)


def _green_error(ppl):
    d = _vacuum_desc(ppl)
    g = Grid(d)
    eps = np.ones((g.nx, g.ny))
    i_f, j_f = g.nx // 2, g.ny // 2
    b = np.zeros((g.nx, g.ny), dtype=complex)
    b[i_f, j_f] = -1.0 / g.h ** 2           # discrete delta of weight -1
    u = Solver(g, eps, refine=0).solve(b)
    I, J = np.meshgrid(np.arange(g.nx), np.arange(g.ny), indexing="ij")
    r = g.h * np.hypot(I - i_f, J - j_f)
    ring = (r >= 1.0) & (r <= 3.0)
    exact = 0.25j * scipy.special.hankel1(0, g.k0 * r[ring])
    return np.max(np.abs(u[ring] - exact)) / np.max(np.abs(exact))


@pytest.mark.slow
def test_vacuum_green_function_second_order():
    e20 = _green_error(20)
    e40 = _green_error(40)
    # O((k h)^2) dispersion error: about 4x smaller per halving of h
    assert e20 < 0.15
    assert 3.0 < e20 / e40 < 5.0


def test_flux_conservation_between_nested_contours():
    # Discrete Green identity for real eps: Im sum_Omega conj(u) b equals the net
    # flux sum over edges leaving Omega of Im(conj(u_in) u_out) / h^2.
    wl = W.small(kind=W.OBJ_POINT)
    g = Grid(wl.grid)
    eps = rasterize_eps(g, W.widths(wl.grid.n_cells, 4))
    b = np.zeros((g.nx, g.ny), dtype=complex)
    b[g.nx // 2, g.j_pillar1 + 5] = 1.0
    b[g.nx // 2 + 7, g.j_src] = 0.3 - 0.2j
    u = Solver(g, eps).solve(b)
    h2 = g.h ** 2

    def flux(i0, i1, j0, j1):           # box [i0, i1) x [j0, j1)
        tot = 0.0
        tot += np.sum(np.imag(np.conj(u[i0, j0:j1]) * u[i0 - 1, j0:j1]))
        tot += np.sum(np.imag(np.conj(u[i1 - 1, j0:j1]) * u[i1, j0:j1]))
        tot += np.sum(np.imag(np.conj(u[i0:i1, j0]) * u[i0:i1, j0 - 1]))
        tot += np.sum(np.imag(np.conj(u[i0:i1, j1 - 1]) * u[i0:i1, j1]))
        return tot / h2

    def emitted(i0, i1, j0, j1):
        return float(np.sum(np.imag(np.conj(u[i0:i1, j0:j1]) * b[i0:i1, j0:j1])))

    p = g.npml
    inner = (p + 3, g.nx - p - 3, p + 1, g.ny - p - 1)
    outer = (p + 1, g.nx - p - 1, p, g.ny - p)
    for box in (inner, outer):
        # outgoing waves (exp(-i omega t), PML absorbing): the sources emit positive
        # power and it all leaves through the contour
        assert emitted(*box) > 0
        assert abs(flux(*box) - emitted(*box)) < 1e-10 * abs(emitted(*box))
    assert abs(flux(*inner) - flux(*outer)) < 1e-10 * abs(flux(*outer))


@pytest.mark.parametrize("theta_deg", [0.0, 40.0, -25.0])
def test_planewave_source_matches_lattice_dispersion(theta_deg):
    # Homogeneous substrate everywhere: a line current sqrt(cos t) exp(i kx x) on one
    # row radiates C exp(i kx x) exp(i q |j - js|) with cos q = 2 - cos(kx h) - k^2 h^2/2
    # and C = b h^2 / (2 i sin q) (one-dimensional lattice Green's function).
    # The aperture is 160 lambda wide so that the edge diffraction at its centre stays
    # below 3%, while a missing sqrt(cos theta) (>= 4.8% at 25 deg) or a wrong phase
    # sign or wavenumber still fails.
    d = W.GridDesc(n_cells=400, ny=96, npml=20, rows_sub=10, rows_pillar=4,
                   eps_pillar=2.1, eps_air=2.1, eps_sub=2.1)
    g = Grid(d)
    th = math.radians(theta_deg)
    b = planewave_source(g, th)
    u = Solver(g, np.full((g.nx, g.ny), 2.1), refine=0).solve(b)
    kx = g.k_sub * math.sin(th)
    cq = 2 - math.cos(kx * g.h) - (g.k_sub * g.h) ** 2 / 2
    q = math.acos(cq)
    C = math.sqrt(math.cos(th)) * g.h ** 2 / (2j * math.sin(q))
    ic = np.arange(g.nx // 2 - 40, g.nx // 2 + 40)
    for dj in (0, 3, 10):
        j = g.j_src + dj
        pred = C * np.exp(1j * kx * g.x(ic)) * np.exp(1j * q * dj)
        err = np.max(np.abs(u[ic, j] - pred)) / abs(C)
        assert err < 3e-2, (dj, err)
