"""GB300 reciprocal incoherent-light evaluator: Python binding of librci.so.

The averaged figure of merit <|w^dag u|^2> of a 2-D metasurface under incoherent light
is computed with one reciprocal frequency-domain solve v = A^{-dag} w and the
quadratic form v^dag W v against the light's cross-correlation (Sec. 4.1, Eq. 7); the
brute-force angle average (Eq. 6) is available on the same factorisation as the
comparison.  All numerical work runs in the CUDA library; this module marshals
arguments (ctypes) and uses PyTorch only for device memory and streams.

Importing the package does not load the library; the first call to ``lib()`` does, and
raises if ``librci.so`` has not been built (``python -m paper_2207_10701_gb300.build``).
There is no CPU fallback.
"""
from paper_2207_10701_gb300.rci import (  # noqa: F401
    Grid, RciError, Info, Server, grid_footprint, lib, qform_toeplitz, qform_toeplitz_noalloc, gauss_legendre,
    kernel_launches, set_wait_limit, measure_peaks, block_inverse, cgemm_batched, EXPORTED, QFORM_NOALLOC_MAX_N,
    OBJ_POINT, OBJ_PLANEWAVE, OBJ_VIRTUAL_FOCUS, OBJ_USER_ROW,
    LIGHT_CONE, LIGHT_ANNULUS, LIGHT_USER_LAGS, LIGHT_TABULATED, FP64, FP32_REFINE,
)
