"""Differentiable averaged intensity and a projected-gradient design loop.

Sec. 4.1 optimises the averaged figure of merit with gradients: the gradient of
v^dag W v is 2 Re(v^dag W dv), and the adjoint method turns dv into one more solve
with the same factorisation.  ``rci_avg_intensity_grad`` does all of that on the GPU;
this module wraps it as a ``torch.autograd.Function`` over the pillar widths and runs
a box-constrained ascent on it.  Each evaluation is set_design + factor + two refined
solves + the quadratic form, all in the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from paper_2207_10701_gb300.rci import Grid, _torch


def _autograd_function():
    torch = _torch()

    class AvgIntensity(torch.autograd.Function):
        """F(widths) with dF/dwidths from the adjoint solve.  widths: 1-D float64 tensor
        (host or device); F is returned as a 0-d float64 tensor on the same device."""

        @staticmethod
        def forward(ctx, widths, grid: Grid, obj, light):
            grid.set_design(widths.detach())
            grid.factor()
            F, grad, info = grid.avg_intensity_grad(obj, light)
            ctx.save_for_backward(torch.from_numpy(grad).to(widths.device))
            ctx.info = info
            return torch.tensor(F, dtype=torch.float64, device=widths.device)

        @staticmethod
        def backward(ctx, g_out):
            (grad,) = ctx.saved_tensors
            return g_out * grad, None, None, None

    return AvgIntensity


_FN = None


def avg_intensity(grid: Grid, widths, obj, light):
    """Differentiable F(widths) (see module docstring)."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(widths, grid, obj, light)


@dataclass
class DesignResult:
    widths: np.ndarray
    history: list = field(default_factory=list)   # F after each accepted step
    steps: list = field(default_factory=list)     # step length used at each iteration
    evaluations: int = 0        # evaluations with gradient
    simt_refactors: int = 0     # of which finished on the FP32 SIMT refactorisation
    fp64_fallbacks: int = 0     # of which finished on the FP64 factorisation
    refine_iters_max: int = 0

    def note(self, info) -> None:
        self.evaluations += 1
        self.simt_refactors += int(info.simt_refactor and not info.fallback)
        self.fp64_fallbacks += int(info.fallback)
        self.refine_iters_max = max(self.refine_iters_max, info.refine_iters)


def optimize(grid: Grid, obj, light, widths0, iters: int = 100, step: float = 0.01,
             lo: float = 0.08, hi: float = 0.36, shrink: float = 0.5) -> DesignResult:
    """Maximise F over widths in [lo, hi] (wavelengths) by projected gradient ascent.

    Each iteration moves every width by at most ``step`` along the normalised gradient
    (w <- clip(w + step * g / max|g|, lo, hi)); a step that lowers F is rejected and
    the step length is multiplied by ``shrink``; an accepted step lets it grow back by
    1/shrink up to the initial value.  Every trial costs one evaluation with gradient."""
    w = np.clip(np.asarray(widths0, dtype=np.float64), lo, hi)
    grid.set_design(w)
    grid.factor()
    F, g, info = grid.avg_intensity_grad(obj, light)
    res = DesignResult(widths=w.copy(), history=[F])
    res.note(info)
    t = step
    for _ in range(iters):
        gmax = float(np.max(np.abs(g)))
        if gmax == 0.0:
            break
        trial = np.clip(w + t * g / gmax, lo, hi)
        grid.set_design(trial)
        grid.factor()
        F1, g1, info = grid.avg_intensity_grad(obj, light)
        res.note(info)
        res.steps.append(t)
        if F1 >= F:
            w, F, g = trial, F1, g1
            res.history.append(F)
            t = min(step, t / shrink)
        else:
            t *= shrink
    res.widths = w
    return res
