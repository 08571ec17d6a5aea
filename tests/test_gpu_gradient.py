"""Parity of the CUDA width gradient (adjoint of Eq. 7, through the C-ABI) with the
FP64 CPU oracle, plus the autograd wrapper and the design loop.

Tolerances: F as for rci_avg_intensity (relative 1e-9 FP64, 1e-8 FP32 + refinement);
the gradient element by element against the largest component at the same levels."""
import numpy as np
import pytest

import workloads as W
from oracle.gradient import avg_intensity_grad as o_grad, rule_lags
from oracle.light import quadrature_rule
from oracle.reciprocal import Evaluation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2207_10701_gb300 as P  # noqa: E402
from paper_2207_10701_gb300.design import avg_intensity, optimize  # noqa: E402

TOL = {P.FP64: 1e-9, P.FP32_REFINE: 1e-8}


def _widths(wl, seed):
    period = wl.grid.cell_px / wl.grid.ppl
    return W.widths(wl.grid.n_cells, seed, lo=0.2 * period, hi=min(0.36, 0.9 * period))


CASES = {
    "tiny_point": lambda: W.tiny(kind=W.OBJ_POINT),
    "tiny_virtual": lambda: W.tiny(kind=W.OBJ_VIRTUAL_FOCUS),
    "small_plane": lambda: W.small(kind=W.OBJ_PLANEWAVE),
    "small_virtual": lambda: W.small(kind=W.OBJ_VIRTUAL_FOCUS),
    # 5-px cells: edges fall at every offset inside a column; PML columns on both sides
    "ragged": lambda: W.Workload("ragged", W.GridDesc(n_cells=7, ny=50, cell_px=5, npml=9,
                                                      rows_sub=7, rows_pillar=9),
                                 W.Objective(kind=W.OBJ_PLANEWAVE, monitor_row=30, theta_out=0.1),
                                 W.Light(W.LIGHT_CONE, c=0.3), 40),
    "one_cell": lambda: W.Workload("one_cell", W.GridDesc(n_cells=1, ny=40, npml=6, rows_sub=5,
                                                          rows_pillar=6),
                                   W.Objective(kind=W.OBJ_POINT, i_f=10, j_f=25),
                                   W.Light(W.LIGHT_ANNULUS, th1=0.1, th2=0.4), 20),
}


def _check(F, grad, F_ref, g_ref, tol):
    assert abs(F - F_ref) <= tol * abs(F_ref), (F, F_ref)
    scale = np.max(np.abs(g_ref))
    err = np.max(np.abs(grad - g_ref))
    assert err <= tol * scale, (err, scale)


@pytest.mark.parametrize("prec", [P.FP64, P.FP32_REFINE])
@pytest.mark.parametrize("name", sorted(CASES))
def test_gradient_matches_oracle(name, prec):
    wl = CASES[name]()
    ws = _widths(wl, 4)
    with P.Grid(wl.grid, prec=prec) as g:
        g.set_design(ws)
        g.factor()
        F, grad, info = g.avg_intensity_grad(wl.objective, wl.light)
        F_plain, _ = g.avg_intensity(wl.objective, wl.light)
    assert F == F_plain                       # same value as the non-gradient call
    F_ref, g_ref, _, _ = o_grad(Evaluation(wl, ws), ws)
    _check(F, grad, F_ref, g_ref, TOL[prec])


def test_gradient_user_lags_equals_rule_gradient():
    # W from a quadrature rule, passed as user lags: the oracle's adjoint with the same
    # lags (which the oracle pins against the brute-force gradient of that rule)
    wl = W.small(kind=W.OBJ_VIRTUAL_FOCUS)
    ws = _widths(wl, 8)
    ev = Evaluation(wl, ws)
    theta, wq = quadrature_rule(wl.light, 24)
    lags = rule_lags(ev.g, theta, wq)
    F_ref, g_ref, _, _ = o_grad(ev, ws, lags=lags)
    with P.Grid(wl.grid, prec=P.FP64) as g:
        g.set_design(ws)
        g.factor()
        F, grad, _ = g.avg_intensity_grad(wl.objective, W.Light(W.LIGHT_USER_LAGS, lags=lags))
    _check(F, grad, F_ref, g_ref, 1e-9)


@pytest.mark.parametrize("prec", [P.FP32_REFINE, P.FP64])
def test_gradient_c4_full_size(prec):
    # the gradient workload at full size: 500 cells, virtual focus 20 wavelengths up,
    # cone of +-15 degrees (oracle: two refined sparse-LU solves, ~20 s of CPU)
    wl = W.c4_gradient()
    ws = W.widths(wl.grid.n_cells, 0)
    with P.Grid(wl.grid, prec=prec) as g:
        g.set_design(ws)
        g.factor()
        F, grad, info = g.avg_intensity_grad(wl.objective, wl.light)
    assert info.rel_residual <= 1e-10
    F_ref, g_ref, _, _ = o_grad(Evaluation(wl, ws), ws)
    _check(F, grad, F_ref, g_ref, TOL[prec])


def test_gradient_is_deterministic_and_needs_a_factor():
    wl = W.small(kind=W.OBJ_PLANEWAVE)
    ws = _widths(wl, 1)
    with P.Grid(wl.grid, prec=P.FP32_REFINE) as g:
        g.set_design(ws)
        with pytest.raises(P.RciError) as e:
            g.avg_intensity_grad(wl.objective, wl.light)
        assert e.value.status == 4            # RCI_ESTATE
        g.factor()
        a = g.avg_intensity_grad(wl.objective, wl.light)
        b = g.avg_intensity_grad(wl.objective, wl.light)
        with pytest.raises(P.RciError):
            g.avg_intensity_grad(wl.objective, W.Light(W.LIGHT_CONE, c=2.0))
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_autograd_function_returns_the_adjoint_gradient():
    wl = W.small(kind=W.OBJ_VIRTUAL_FOCUS)
    ws = _widths(wl, 6)
    with P.Grid(wl.grid, prec=P.FP64) as g:
        w = torch.tensor(ws, dtype=torch.float64, device="cuda", requires_grad=True)
        F = avg_intensity(g, w, wl.objective, wl.light)
        (2.5 * F).backward()
        g.set_design(ws)
        g.factor()
        F2, grad, _ = g.avg_intensity_grad(wl.objective, wl.light)
    assert F.item() == F2
    assert torch.equal(w.grad.cpu(), torch.from_numpy(2.5 * grad))


def test_design_loop_ascends_within_bounds():
    wl = W.small(kind=W.OBJ_PLANEWAVE)
    ws = W.widths(wl.grid.n_cells, 3)
    with P.Grid(wl.grid, prec=P.FP32_REFINE) as g:
        res = optimize(g, wl.objective, wl.light, ws, iters=8, step=0.01)
        g.set_design(res.widths)
        g.factor()
        F_end, _ = g.avg_intensity(wl.objective, wl.light)
    h = np.array(res.history)
    assert len(h) >= 2 and np.all(np.diff(h) >= 0) and h[-1] > h[0]
    assert F_end == pytest.approx(h[-1], rel=1e-12)
    assert np.all(res.widths >= 0.08) and np.all(res.widths <= 0.36)


def _edge_clear(ws, idx, h=0.05, margin=2.5e-4):
    """Nudge the widths idx so that both edges sit >= margin from every column boundary
    (then F is smooth in each width over +-margin and central differences apply)."""
    ws = ws.copy()
    for m in idx:
        r = np.mod(ws[m] / 2, h)
        if r < margin or r > h - margin:
            ws[m] += 4 * margin
    return ws


@pytest.mark.parametrize("prec", [P.FP32_REFINE, P.FP64])
def test_gradient_c4_central_differences_on_20_widths(prec):
    # The gradient workload at full size; central differences with h = 1e-4 wavelengths on
    # 20 seeded widths, each a fresh set_design + factor + evaluation on the GPU.  Their
    # O(h^2) truncation error is what separates them from the adjoint gradient: it must
    # fall fourfold when h is halved, and the Richardson combination of h and h/2 removes it.
    wl = W.c4_gradient()
    rng = np.random.default_rng(20)
    idx = np.sort(rng.choice(wl.grid.n_cells, 20, replace=False))
    ws = _edge_clear(W.widths(wl.grid.n_cells, 5), idx)
    with P.Grid(wl.grid, prec=prec) as g:
        # F to ~1e-13 so that its rounding (/ 2 h) stays far below the truncation error
        g.set_refinement(1e-13, 30)
        g.set_design(ws)
        g.factor()
        F, grad, _ = g.avg_intensity_grad(wl.objective, wl.light)
        fd = {}
        for step in (1e-4, 5e-5):
            d = np.empty(len(idx))
            for t, m in enumerate(idx):
                vals = []
                for sgn in (1, -1):
                    w = ws.copy()
                    w[m] += sgn * step
                    g.set_design(w)
                    g.factor()
                    vals.append(g.avg_intensity(wl.objective, wl.light)[0])
                d[t] = (vals[0] - vals[1]) / (2 * step)
            fd[step] = d
    scale = np.max(np.abs(grad))
    e1 = np.max(np.abs(fd[1e-4] - grad[idx]))
    e2 = np.max(np.abs(fd[5e-5] - grad[idx]))
    rich = (4 * fd[5e-5] - fd[1e-4]) / 3
    assert e1 <= 3e-5 * scale, (e1, scale)
    assert 3.5 <= e1 / e2 <= 4.5, (e1, e2)
    assert np.max(np.abs(rich - grad[idx])) <= 1e-7 * scale


def test_gradient_c4_against_oracle_bruteforce_gradient():
    # full size: the adjoint gradient for the Toeplitz W of a 12-point rule against the
    # oracle's gradient of the brute-force average over the same 12 angles (the two are
    # equal up to rounding for a rule symmetric in theta)
    from oracle.gradient import bruteforce_grad
    wl = W.c4_gradient()
    ws = W.widths(wl.grid.n_cells, 9)
    ev = Evaluation(wl, ws)
    theta, wq = quadrature_rule(wl.light, 12)
    F_bf, g_bf = bruteforce_grad(ev, ws, theta, wq)
    lags = rule_lags(ev.g, theta, wq)
    with P.Grid(wl.grid, prec=P.FP32_REFINE) as g:
        g.set_design(ws)
        g.factor()
        F, grad, _ = g.avg_intensity_grad(wl.objective, W.Light(W.LIGHT_USER_LAGS, lags=lags))
    _check(F, grad, F_bf, g_bf, 1e-8)


def test_design_loop_c4_100_iterations():
    # 100 projected-gradient iterations on the full gradient workload, FP32 + refinement
    wl = W.c4_gradient()
    ws = W.widths(wl.grid.n_cells, 0)
    with P.Grid(wl.grid, prec=P.FP32_REFINE) as g:
        res = optimize(g, wl.objective, wl.light, ws, iters=100, step=0.01)
    h = np.array(res.history)
    assert len(res.steps) == 100
    assert np.all(np.diff(h) >= 0) and h[-1] > h[0], (h[0], h[-1], len(h))
    assert np.all(res.widths >= 0.08) and np.all(res.widths <= 0.36)
    # every evaluation of the ascent finishes in FP32 (plain or Krylov refinement)
    assert res.evaluations == 101 and res.fp64_fallbacks == 0, res
