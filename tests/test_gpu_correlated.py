"""Parity of the correlated-light, dense-W and multi-output forms (through the C-ABI) with
the FP64 oracle.  Tolerances as for rci_avg_intensity: relative 1e-9 (FP64) and 1e-8
(FP32 + refinement) on F."""
import numpy as np
import pytest

import workloads as W
from oracle.correlated import avg_intensity_correlated as o_corr, avg_intensity_multi as o_multi
from oracle.correlated import correlated_W
from oracle.gradient import rule_lags
from oracle.light import quadrature_rule
from oracle.reciprocal import Evaluation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2207_10701_gb300 as P  # noqa: E402

TOL = {P.FP64: 1e-9, P.FP32_REFINE: 1e-8}


def _widths(wl, seed):
    period = wl.grid.cell_px / wl.grid.ppl
    return W.widths(wl.grid.n_cells, seed, lo=0.2 * period, hi=min(0.36, 0.9 * period))


def _hermitian_psd(seed, n):
    rng = np.random.default_rng(seed)
    G = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return G @ G.conj().T / n


def _rule(seed, n, c):
    rng = np.random.default_rng(seed)
    return np.sort(rng.uniform(-c, c, n)), rng.uniform(0.05, 0.2, n)


CASES = {
    "tiny_point": lambda: W.tiny(kind=W.OBJ_POINT),
    "tiny_virtual": lambda: W.tiny(kind=W.OBJ_VIRTUAL_FOCUS),
    "small_plane": lambda: W.small(kind=W.OBJ_PLANEWAVE),
    "small_virtual": lambda: W.small(kind=W.OBJ_VIRTUAL_FOCUS),
}


@pytest.mark.parametrize("prec", [P.FP64, P.FP32_REFINE])
@pytest.mark.parametrize("name", sorted(CASES))
def test_correlated_matches_oracle(name, prec):
    wl = CASES[name]()
    ws = _widths(wl, 2)
    theta, om = _rule(3, 11, 0.6)
    C = _hermitian_psd(4, 11)
    with P.Grid(wl.grid, prec=prec) as g:
        g.set_design(ws)
        g.factor()
        F, _ = g.avg_intensity_correlated(wl.objective, theta, om, C)
    F_ref = o_corr(Evaluation(wl, ws), theta, om, C)
    assert abs(F - F_ref) <= TOL[prec] * abs(F_ref), (F, F_ref)


def test_diagonal_correlation_equals_gpu_brute_force_and_rule_lags():
    wl = W.small(kind=W.OBJ_VIRTUAL_FOCUS)
    ws = _widths(wl, 5)
    theta, wq = quadrature_rule(wl.light, 16)
    with P.Grid(wl.grid, prec=P.FP64) as g:
        g.set_design(ws)
        g.factor()
        Fc, _ = g.avg_intensity_correlated(wl.objective, theta, np.sqrt(wq), np.eye(16))
        Fb, _, _ = g.solve_angles(wl.objective, theta, wq)               # forward, 16 solves
        lags = rule_lags(Evaluation(wl, ws).g, theta, wq)
        Fl, _ = g.avg_intensity(wl.objective, W.Light(W.LIGHT_USER_LAGS, lags=lags))
    assert Fc == pytest.approx(Fb, rel=1e-9)
    assert Fc == pytest.approx(Fl, rel=1e-12)


@pytest.mark.parametrize("prec", [P.FP64, P.FP32_REFINE])
def test_dense_form_matches_correlated_and_oracle(prec):
    wl = W.small(kind=W.OBJ_PLANEWAVE)
    ws = _widths(wl, 7)
    ev = Evaluation(wl, ws)
    theta, om = _rule(8, 9, 0.5)
    C = _hermitian_psd(9, 9)
    Wd = torch.from_numpy(correlated_W(ev.g, theta, om, C)).cuda()
    with P.Grid(wl.grid, prec=prec) as g:
        g.set_design(ws)
        g.factor()
        Fd, _ = g.avg_intensity_dense(wl.objective, Wd)
        Fc, _ = g.avg_intensity_correlated(wl.objective, theta, om, C)
    assert Fd == pytest.approx(Fc, rel=1e-11)
    F_ref = o_corr(ev, theta, om, C)
    assert abs(Fd - F_ref) <= TOL[prec] * abs(F_ref)


@pytest.mark.parametrize("prec", [P.FP64, P.FP32_REFINE])
def test_multi_output_matches_single_and_oracle(prec):
    wl = W.small(kind=W.OBJ_PLANEWAVE)
    ws = _widths(wl, 11)
    top = wl.objective.monitor_row
    nx = wl.grid.n_cells * wl.grid.cell_px + 2 * wl.grid.npml
    objs = [W.Objective(kind=W.OBJ_PLANEWAVE, monitor_row=top, theta_out=t) for t in (0.0, 0.07, -0.12)]
    objs += [W.Objective(kind=W.OBJ_POINT, i_f=nx // 2, j_f=top + 3),
             W.Objective(kind=W.OBJ_VIRTUAL_FOCUS, monitor_row=top, x_f=1.0, d_rows=25)]
    with P.Grid(wl.grid, prec=prec) as g:
        g.set_design(ws)
        g.factor()
        Fm, tot, _ = g.avg_intensity_multi(objs, wl.light)
        single = [g.avg_intensity(o, wl.light)[0] for o in objs]
    ev = Evaluation(wl, ws)
    ref = o_multi(ev, objs, ev.lags())
    for F, Fs, Fr in zip(Fm, single, ref):
        assert abs(F - Fs) <= TOL[prec] * abs(Fs)
        assert abs(F - Fr) <= TOL[prec] * abs(Fr)
    assert tot == pytest.approx(float(np.sum(Fm)), rel=1e-15)


def test_multi_output_crosses_the_chunk_boundary():
    wl = W.tiny(kind=W.OBJ_PLANEWAVE)
    ws = _widths(wl, 12)
    top = wl.objective.monitor_row
    angles = np.linspace(-0.3, 0.3, 300)
    objs = [W.Objective(kind=W.OBJ_PLANEWAVE, monitor_row=top, theta_out=float(t)) for t in angles]
    with P.Grid(wl.grid, prec=P.FP64) as g:
        g.set_design(ws)
        g.factor()
        Fm, _, _ = g.avg_intensity_multi(objs, wl.light)
        for k in (0, 255, 256, 299):
            Fs, _ = g.avg_intensity(objs[k], wl.light)
            assert Fm[k] == pytest.approx(Fs, rel=1e-9)


def test_correlated_c2_full_size():
    # the 200-wavelength collimator with a random correlation on a 48-point annulus rule
    wl = W.c2_collimator()
    ws = W.widths(wl.grid.n_cells, 3)
    theta, wq = quadrature_rule(wl.light, 48)
    C = _hermitian_psd(13, 48)
    with P.Grid(wl.grid, prec=P.FP32_REFINE) as g:
        g.set_design(ws)
        g.factor()
        F, info = g.avg_intensity_correlated(wl.objective, theta, np.sqrt(wq), C)
    F_ref = o_corr(Evaluation(wl, ws), theta, np.sqrt(wq), C)
    assert abs(F - F_ref) <= 1e-8 * abs(F_ref)
