"""Write the oracle's values for the full-size virtual-focus workloads (test fixtures).

For each (workload, design seed) below this runs the FP64 CPU oracle -- and nothing
else -- on the full grid and stores, in <workload>_seed<seed>.json beside this script:

  F          the averaged intensity of Eq. 7, v^dag W v, from the refined oracle solve
  v_idx, v   the reciprocal field on the source plane at 257 evenly spaced interior
             columns (complex, as [re, im] pairs)
  v_norm2    ||v||_2 over the whole source plane
  rel_residual   ||b - A z||_2 / ||b||_2 of the oracle's field, in double-double
  seconds    wall time of the oracle evaluation

The GPU parity tests compare the library's F and v with these values; the bench line
reports its full-size precision-form error against them.  Regenerate with

    python tests/golden/make_golden.py            (about 2 minutes and 15 GB per C3 design)
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle.grid import objective_vector  # noqa: E402
from oracle.reciprocal import Evaluation, qform_direct, source_plane  # noqa: E402
from oracle.solve import residual_dd  # noqa: E402

CASES = [("c3_precision", 21), ("c3_precision", 0), ("c4_gradient", 21)]


def golden(name: str, seed: int) -> dict:
    wl = W.WORKLOADS[name]()
    ws = W.widths(wl.grid.n_cells, seed)
    t0 = time.perf_counter()
    ev = Evaluation(wl, ws)
    b = np.conj(objective_vector(ev.g, wl.objective))
    z = ev.solver.solve(b)
    v = source_plane(ev.g, np.conj(z))
    F = qform_direct(v, ev.lags())
    secs = time.perf_counter() - t0
    r = residual_dd(ev.solver.coeffs, b, z)
    idx = np.unique(np.linspace(0, v.size - 1, 257).round().astype(int))
    return {
        "workload": name, "seed": seed, "n_cells": wl.grid.n_cells, "ny": wl.grid.ny,
        "unknowns": int(ev.g.N), "n_src": int(v.size), "F": F,
        "v_idx": idx.tolist(), "v": [[float(c.real), float(c.imag)] for c in v[idx]],
        "v_norm2": float(np.linalg.norm(v)),
        "rel_residual": float(np.linalg.norm(r) / np.linalg.norm(b)),
        "seconds": round(secs, 1),
        "command": "python tests/golden/make_golden.py",
    }


def path(name: str, seed: int) -> str:
    return os.path.join(HERE, f"{name}_seed{seed}.json")


def main(argv):
    todo = CASES if not argv else [c for c in CASES if f"{c[0]}_seed{c[1]}" in argv]
    for name, seed in todo:
        d = golden(name, seed)
        with open(path(name, seed), "w") as f:
            json.dump(d, f, indent=1)
            f.write("\n")
        print(f"{name} seed {seed}: F = {d['F']:.16e}  residual {d['rel_residual']:.2e}  "
              f"({d['seconds']} s)", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
