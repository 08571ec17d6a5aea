"""One evaluation case to run under a profiler (ncu launch lists and kernel captures).

    python -m paper_2207_10701_gb300.profile_case --cells 500 --prec fp32 --repeat 2

builds the grid of an n-cell metasurface (ny = 160 by default, the 200-wavelength
collimator's height), then `repeat` times: set a seeded design, factor, and evaluate the
averaged intensity of a 10-30 degree annulus on a 0-degree planewave mode (with
--grad, the adjoint gradient as well).  Everything runs in librci.so; the script only
sets the case up, so the kernels a profiler sees are exactly the library's.
"""
from __future__ import annotations

import argparse

import workloads as W
import paper_2207_10701_gb300 as P


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, default=500)
    ap.add_argument("--ny", type=int, default=160)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--grad", action="store_true")
    a = ap.parse_args(argv)
    d = W.GridDesc(n_cells=a.cells, ny=a.ny)
    prec = P.FP64 if a.prec == "fp64" else P.FP32_REFINE
    obj = W.Objective(kind=W.OBJ_PLANEWAVE, monitor_row=d.npml + d.rows_sub + d.rows_pillar + 10)
    light = W.Light(W.LIGHT_ANNULUS, th1=W.deg(10), th2=W.deg(30))
    with P.Grid(d, prec=prec) as g:
        for r in range(a.repeat):
            g.set_design(W.widths(d.n_cells, r))
            g.factor()
            if a.grad:
                F, _, info = g.avg_intensity_grad(obj, light)
            else:
                F, info = g.avg_intensity(obj, light)
            print(f"case {r}: F = {F:.12e}, refinement steps {info.refine_iters}, "
                  f"rel. residual {info.rel_residual:.2e}")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
