"""Refinement of hard designs on the GPU.  A design of the serving stream on which plain
refinement with the FP32 factorisation stalls (a step reducing the residual less than
0.7-fold) is finished by flexible GMRES preconditioned by the FP32 solve instead of the FP64
fallback; a design whose tensor-core FP32 factorisation (3xTF32 products) cannot resolve it
at all is factored again on the FP32 SIMT pipe before any FP64 work.  In both cases the
averaged intensity (Eq. 7) matches the FP64 oracle's."""
import numpy as np
import pytest

import workloads as W
from oracle.reciprocal import Evaluation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2207_10701_gb300 as P  # noqa: E402

# request 32 of the 512-request serving stream (seed 1, a quarter repeated designs): 253
# cells, ny 160, growth estimate about 51; plain refinement stalls after its second step
STALL_REQUEST = 32
# request 243 of the same stream: 1075 cells (nx 8640), growth estimate about 50; the
# tensor-core FP32 factorisation gives a non-finite solve, the FP32 SIMT one a solve that
# refinement (with Krylov steps) takes to the tolerance
SIMT_REQUEST = 243


def _request(k=STALL_REQUEST):
    return W.serving_requests(512, 50.0, seed=1, repeat_fraction=0.25)[k]


def test_krylov_refinement_finishes_a_stalled_solve_and_matches_the_oracle():
    r = _request()
    with P.Grid(r.grid, prec=P.FP32_REFINE) as g:
        g.set_design(r.widths)
        g.factor()
        F, info = g.avg_intensity(r.objective, r.light)
    assert info.krylov_steps > 0, "plain refinement converged: this design no longer stalls"
    assert not info.fallback
    assert info.rel_residual <= 1e-10
    wl = W.Workload("serving-32", r.grid, r.objective, r.light, n_angles=0)
    F_ref, _ = Evaluation(wl, r.widths).reciprocal()
    assert abs(F - F_ref) <= 1e-8 * abs(F_ref), (F, F_ref)


def test_krylov_refinement_respects_the_step_budget():
    # with a budget that plain refinement alone uses up, no Krylov step is taken and the
    # design finishes on the FP64 fallback, as before
    r = _request()
    with P.Grid(r.grid, prec=P.FP32_REFINE) as g:
        g.set_refinement(1e-10, 2)
        g.set_design(r.widths)
        g.factor()
        F, info = g.avg_intensity(r.objective, r.light)
    assert info.krylov_steps == 0
    assert info.fallback and info.simt_refactor  # the SIMT rung ran, then the FP64 one
    assert np.isfinite(F)


def test_simt_refactor_resolves_a_design_the_tensor_core_factorisation_cannot():
    r = _request(SIMT_REQUEST)
    with P.Grid(r.grid, prec=P.FP32_REFINE) as g:
        g.set_design(r.widths)
        g.factor()
        F, info = g.avg_intensity(r.objective, r.light)
        assert info.simt_refactor, "the tensor-core factorisation now resolves this design"
        assert not info.fallback
        assert info.rel_residual <= 1e-10
        # a new design starts on the tensor-core factorisation again
        g.set_design(W.widths(r.grid.n_cells, 7))
        g.factor()
        _, info2 = g.avg_intensity(r.objective, r.light)
        assert not info2.simt_refactor and not info2.fallback, info2
    wl = W.Workload("serving-243", r.grid, r.objective, r.light, n_angles=0)
    F_ref, _ = Evaluation(wl, r.widths).reciprocal()
    assert abs(F - F_ref) <= 1e-8 * abs(F_ref), (F, F_ref)
