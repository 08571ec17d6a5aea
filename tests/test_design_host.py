"""Host bookkeeping of the design loop (no GPU): how the evaluations of an ascent finished,
as `bench.py` reports them — the SIMT rung counted only when it resolved the design, the FP64
fallback whenever it ran, the largest refinement count."""
import paper_2207_10701_gb300 as P
from paper_2207_10701_gb300.design import DesignResult


def _info(iters, fallback=False, simt=False):
    return P.Info(iters, 1e-11, 0.0, 0.0, 0.0, fallback, 1.0, 0, simt)


def test_design_result_counts_how_evaluations_finished():
    res = DesignResult(widths=None)
    for info in (_info(2), _info(9), _info(4, simt=True), _info(1, fallback=True, simt=True)):
        res.note(info)
    assert res.evaluations == 4
    assert res.simt_refactors == 1          # the SIMT rung that had to hand over to FP64 excluded
    assert res.fp64_fallbacks == 1
    assert res.refine_iters_max == 9
