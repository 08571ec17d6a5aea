"""Failure detection on the GPU without a fault: a tensor-core pipeline wait that runs out.

Every wait of the tensor-core kernels is bounded.  Lowering the bound to a few hundred
cycles makes the first wait on an operand stage run out; the kernel then records a device
status (no trap), waits at the full bound for its own tensor-core operations, frees its
tensor memory and returns, so the context stays usable.  rci_factor reports RCI_ETIMEOUT,
and with the default bound restored the same grid factors and evaluates as before."""
import numpy as np
import pytest

import workloads as W
from oracle.reciprocal import Evaluation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2207_10701_gb300 as P  # noqa: E402

RCI_ETIMEOUT = 8


def test_expired_tensor_core_wait_is_reported_and_the_grid_recovers():
    wl = W.c1_concentrator()                 # level 1: 110 products of 128^3 on tcgen05
    ws = W.widths(wl.grid.n_cells, 3)
    F_ref, _ = Evaluation(wl, ws).reciprocal()
    with P.Grid(wl.grid, prec=P.FP32_REFINE) as g:
        g.set_design(ws)
        old = P.set_wait_limit(300)
        try:
            with pytest.raises(P.RciError) as ei:
                g.factor()
            assert ei.value.status == RCI_ETIMEOUT
        finally:
            P.set_wait_limit(0)              # default bound again
        assert old > 1e9
        with pytest.raises(P.RciError):      # a timed-out factorisation is not usable
            g.avg_intensity(wl.objective, wl.light)
        g.factor()
        F, info = g.avg_intensity(wl.objective, wl.light)
    assert abs(F - F_ref) <= 1e-8 * F_ref, (F, F_ref, info)
    assert np.isfinite(F)
