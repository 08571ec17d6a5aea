"""CPU oracle for the reciprocal incoherent-light evaluation (TEST INFRASTRUCTURE ONLY).

Plain, slow, FP64 restatement of what the method computes, written from the paper
(Pestourie, Yao, Kante & Johnson, "Efficient inverse design of large-area metasurfaces
for incoherent light"), used only by the tests, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product path (the CUDA
library and its Python binding) never imports, links or executes anything here, and this
package imports nothing from the product package.  Only the seeded input descriptions in
``workloads`` are shared.

Modules
  grid        geometry, PML stretch, permittivity raster, FDFD operator A (Sec. 4.1),
              equivalent planewave currents b0(theta) (Sec. 3, Sec. 4.1) and objective
              vectors w (Sec. 4.1), virtual-focus lattice propagator.
  solve       u = A^{-1} b with a library sparse LU as the solve step, then iterative
              refinement with a double-double residual.
  light       angular densities, cross-correlation W (Eq. 4, annulus formula of
              Sec. 5.1, in the exact reading), Gauss-Legendre rules (Sec. 5.2).
  reciprocal  reciprocal average v^dag W v (Eq. 7), brute-force angle average (Eq. 6),
              FFT and spectral forms of the quadratic form.
  gradient    dF/d(widths) by the adjoint of v^dag W v (Sec. 4.1), the brute-force
              gradient of Eq. 6 angle by angle, and the derivative of the fill raster.
  correlated  correlated incoherent light (the W of Eq. 3 on a quadrature, the forward
              double sum of Eq. 5), dense v^dag W v, multi-output objectives (Sec. 6).

Every function is pinned by a ``-m "not gpu"`` test against something other than
itself (closed forms, library routines used as independent checks, invariants, the
exact discrete identity behind Eq. 7).  No function is parity-unpinned.
"""
