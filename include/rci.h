/*
 * rci.h -- C ABI of the GB300 reciprocal incoherent-light evaluator.
 *
 * The library computes the average figure of merit <|w^dag u|^2> of a 2-D
 * metasurface under incoherent light with a single "reciprocal" frequency-domain
 * solve v = A^{-dag} w followed by the quadratic form v^dag W v against the
 * light's cross-correlation W (paper Sec. 4.1, Eq. 7), and, as the in-run
 * comparison, the brute-force angle average of Eq. 6 as a multi-right-hand-side
 * solve on the same factorisation (Sec. 5.2).
 *
 * Discretisation (the paper keeps the operator abstract, Sec. 4.1; this is the
 * library's reading): scalar Helmholtz at wavelength 1 on a uniform grid
 * h = 1/ppl, stretched-coordinate PML on all four sides, multiplied by s_x s_y so
 * that A is complex symmetric (A = A^T).  Unknowns are ordered k = i*ny + j (x
 * outermost), which makes A block tridiagonal along the metasurface with
 * tridiagonal ny x ny diagonal blocks and diagonal couplings.
 *   node (i, j): x_i = (i - npml + 1/2) h, y_j = (j + 1/2) h
 *   nx = n_cells*cell_px + 2*npml; interior columns S = [npml, nx - npml), n_src = |S|
 *   source row j_src = npml + src_offset; pillars in rows
 *   [npml + rows_sub, npml + rows_sub + rows_pillar); substrate below, air above.
 *
 * Memory and ownership.  A grid owns all of its device memory (allocated at
 * rci_create_grid / first use, released by rci_destroy_grid).  The caller owns
 * every buffer it passes.  Each pointer argument states whether it is HOST or
 * DEVICE memory.  Complex vectors are interleaved (re, im) float64 pairs.
 *
 * Streams.  All device work of a grid runs on the stream given at creation
 * (NULL = legacy default stream).  Calls that return a host scalar synchronise
 * that stream before returning.  A grid must not be used by two host threads
 * at once.
 *
 * Errors.  Every call returns an rci_status.  Outputs are written only on
 * RCI_OK, except RCI_ENOCONV, which still returns the best value reached (with
 * the info record filled).  rci_last_error() gives a message for the last
 * failure on a grid.  No exception crosses the ABI.
 */
#ifndef RCI_H
#define RCI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RCI_OK = 0,
  RCI_EINVAL = 1,     /* bad argument or size */
  RCI_ENOMEM = 2,     /* device allocation failed */
  RCI_ECUDA = 3,      /* a CUDA call failed */
  RCI_ESTATE = 4,     /* call out of order (no design, not factored) */
  RCI_ESINGULAR = 5,  /* zero pivot in a block inversion */
  RCI_ENOCONV = 6,    /* iterative refinement did not reach the tolerance */
  RCI_ENUMERIC = 7,   /* NaN or Inf in an input or result */
  RCI_ETIMEOUT = 8    /* a bounded device wait expired */
} rci_status;

typedef enum {
  RCI_FP64 = 0,        /* factor, solve and residual in FP64 */
  RCI_FP32_REFINE = 1  /* factor and solve in FP32, FP64 stencil residual refinement */
} rci_precision;

typedef enum {
  RCI_OBJ_POINT = 0,          /* concentrator, focus on node (i_f, j_f): w = e_f */
  RCI_OBJ_PLANEWAVE = 1,      /* collimator: w_i = exp(i k0 sin(theta_out) x_i) on monitor_row, i in S */
  RCI_OBJ_VIRTUAL_FOCUS = 2,  /* concentrator, focus d_rows above monitor_row at x_f:
                                 w_i = conj(K(x_f - x_i)) on monitor_row, i in S, with K the
                                 lattice propagator through homogeneous air (see rci_solve_reciprocal) */
  RCI_OBJ_USER_ROW = 3        /* w given by the caller on monitor_row, i in S */
} rci_objective_kind;

typedef enum {
  RCI_LIGHT_CONE = 0,       /* rho uniform in theta on [-c, c] */
  RCI_LIGHT_ANNULUS = 1,    /* rho uniform in theta on [th1, th2] U [-th2, -th1] */
  RCI_LIGHT_USER_LAGS = 2,  /* real, even W given as lags W(m h), m = 0..n_src-1 */
  RCI_LIGHT_TABULATED = 3   /* rho given at angles: piecewise linear in theta, even (below) */
} rci_light_kind;

/* Problem geometry (lengths in wavelengths, counts in grid cells). */
typedef struct {
  int32_t n_cells;      /* unit cells (one pillar each) */
  int32_t ny;           /* rows, PML included: 4 .. 256 (the single-right-hand-side solve
                           holds a row of the stored blocks in registers); even for FP32_REFINE
                           (rows are read as pairs of complex64) */
  int32_t ppl;          /* grid points per wavelength, h = 1/ppl */
  int32_t cell_px;      /* unit-cell period in cells */
  int32_t npml;         /* PML thickness in cells on all four sides */
  int32_t rows_sub;     /* substrate rows between the bottom PML and the pillars */
  int32_t rows_pillar;  /* pillar height in rows */
  int32_t src_offset;   /* source row = npml + src_offset */
  double eps_pillar, eps_sub, eps_air;
  double pml_R0;        /* PML normal-incidence reflection target, sigma_max = -(m+1) ln(R0) / (2 d) */
  int32_t pml_m;        /* PML polynomial grading order */
  int32_t prec;         /* rci_precision */
  int32_t device;       /* CUDA device ordinal */
  int32_t reserved;
} rci_grid_desc;

typedef struct {
  int32_t kind;          /* rci_objective_kind */
  int32_t monitor_row;   /* PLANEWAVE / VIRTUAL_FOCUS / USER_ROW */
  int32_t i_f, j_f;      /* POINT */
  double theta_out;      /* PLANEWAVE: output angle in air (radians) */
  double x_f;            /* VIRTUAL_FOCUS: focus abscissa (wavelengths) */
  int32_t d_rows;        /* VIRTUAL_FOCUS: focus height above monitor_row (rows, >= 0) */
  int32_t reserved;
  const double* w_row;   /* USER_ROW: HOST complex128[n_src] (interleaved) */
} rci_objective;

typedef struct {
  int32_t kind;          /* rci_light_kind */
  int32_t reserved;
  double c;              /* CONE half-angle (radians, 0 < c < pi/2) */
  double th1, th2;       /* ANNULUS bounds (0 <= th1 < th2 < pi/2) */
  const double* lags;    /* USER_LAGS: HOST float64[n_src] */
  /* TABULATED: the angular density (Sec. 3's <|a(theta)|^2>) at n_tab angles
   * 0 <= theta[0] < theta[1] < ... < theta[n_tab-1] < pi/2 (radians, in the substrate),
   * rho[q] >= 0, linear in theta between nodes, zero outside [theta[0], theta[n_tab-1]] and
   * even (rho(-theta) = rho(theta)), so that
   *   W(D) = 2 int rho(theta) cos(theta) cos(k_s sin(theta) D) dtheta,
   * evaluated on the device by composite Gauss-Legendre quadrature in u = sin(theta) on
   * sub-panels no wider than half an oscillation period over the source plane.  The values
   * are used as given (no normalisation).  HOST float64[n_tab] each, 2 <= n_tab <= 65536. */
  const double* tab_theta;
  const double* tab_rho;
  int64_t n_tab;
} rci_light;

typedef struct {
  int32_t refine_iters;  /* refinement steps taken by the last solve */
  int32_t fallback;      /* 1: an FP32_REFINE grid finished the solve on its FP64 fallback
                            factorisation (see rci_set_refinement) */
  double rel_residual;   /* ||b - A x||_2 / ||b||_2 after the last solve (FP64 stencil) */
  double ms_factor;      /* device time of the last factorisation */
  double ms_solve;       /* device time of the last solve incl. refinement */
  double ms_qform;       /* device time of the last quadratic form */
  double growth_est;     /* growth estimate of the factorisation used: the largest |re|, |im|
                            among the diagonal blocks it inverted (the Schur complements of every
                            reduction level) over the largest among A's coefficients.  Block
                            cyclic reduction pivots only inside blocks, so large values flag a
                            factorisation whose rounding errors refinement must absorb. */
  int32_t krylov_steps;  /* FP32_REFINE: preconditioned steps of the Krylov refinement taken
                            after plain refinement stalled (0: plain refinement sufficed);
                            they are included in refine_iters */
  int32_t simt_refactor; /* FP32_REFINE: 1 when the design was factored again on the FP32 SIMT
                            pipe because its tensor-core factorisation could not resolve it
                            (see rci_set_refinement); refine_iters and krylov_steps are then
                            those of the solve on that factorisation */
} rci_info;

typedef struct rci_grid rci_grid;

/* Create a grid for one geometry on one device.  stream: cudaStream_t or NULL.
 * Allocates the operator and factor storage for the descriptor's size.
 * Errors: EINVAL (bad descriptor), ENOMEM, ECUDA. */
rci_status rci_create_grid(const rci_grid_desc* desc, void* stream, rci_grid** out);

/* Release every device allocation of the grid.  NULL is accepted. */
rci_status rci_destroy_grid(rci_grid* g);

/* Sizes and device footprint.  Any output pointer may be NULL. HOST outputs. */
rci_status rci_grid_query(const rci_grid* g, int64_t* nx, int64_t* ny, int64_t* n_src,
                          size_t* device_bytes);

/* Set the pillar widths (wavelengths, one per cell, each in (0, period)) and
 * assemble A: permittivity raster (area-weighted fill per column in the pillar
 * rows) and the stretched-coordinate stencil.  Invalidates the factorisation.
 * widths: HOST or DEVICE float64[n_cells] as widths_on_device says.  Host widths
 * outside (0, period) fail here with EINVAL; device widths are checked on the device
 * and the next rci_factor fails with EINVAL (the call itself does not synchronise). */
rci_status rci_set_design(rci_grid* g, const double* widths, int64_t n_cells, int widths_on_device);

/* Factor A by block cyclic reduction along x (the direct solver behind every
 * solve; Sec. 4.1 asks for one solve per evaluation).  Precision per grid.  An
 * FP32_REFINE grid whose factorisation meets a zero pivot factors the design again on
 * the FP32 SIMT pipe and, if a pivot vanishes there too, in FP64 (rci_set_refinement).
 * Errors: ESTATE (no design), ESINGULAR (zero pivot in a diagonal block of the FP64
 * factorisation), EINVAL (a device width out of range), ETIMEOUT (an expired bounded
 * wait of a tensor-core kernel). */
rci_status rci_factor(rci_grid* g);

/* Solve A x = b for nrhs right-hand sides stored [i][j][q] (q fastest):
 * b, x: DEVICE complex128[nx*ny*nrhs].  x may alias b.  FP32_REFINE grids refine
 * every right-hand side with the FP64 stencil residual to the grid's tolerance (rel.
 * residual 1e-10 by default, rci_set_refinement);
 * FP64 grids take up to two refinement steps.  info (HOST, may be NULL). */
rci_status rci_solve(rci_grid* g, const double* b, double* x, int64_t nrhs, rci_info* info);

/* Iterative refinement settings of the grid: stop when ||b - A x||_2 / ||b||_2 <= tol
 * (FP64 stencil residual) or after max_steps corrections (the first FP32 solve is not
 * counted).  Defaults: FP32_REFINE tol 1e-10, 30 steps; FP64 tol 1e-13, 2 steps.
 * When plain refinement of a single right-hand side stalls (a step that reduces the
 * residual less than 0.7-fold, after the second, or max_steps steps), it continues with
 * flexible GMRES on the FP64 stencil operator preconditioned by the FP32 factorisation
 * (restarted every 16 steps; each step one FP32 solve, counted in the same max_steps
 * budget; rci_info.krylov_steps).
 * An FP32_REFINE grid whose refinement fails -- a non-finite residual, plain and Krylov
 * refinement both stalled or out of steps, or a zero FP32 pivot in rci_factor -- first
 * factors the current design again in FP32 on the SIMT pipe (one rounding per FMA where
 * the tensor-core factorisation rounds its 3xTF32 products about 3.5 times more coarsely)
 * and repeats the solve on it (rci_info.simt_refactor); if that fails too, it factors the
 * design once in FP64
 * (the FP64 factor store is allocated the first time, from the grid's memory source)
 * and finishes this and every later solve of that design on it (rci_info.fallback).
 * The next rci_set_design returns the grid to the tensor-core factorisation.
 * A solve that ends above tol returns RCI_ENOCONV with its best value (FP64 and fallback
 * solves only above 1e-9).  tol > 0, 0 <= max_steps <= 100. */
rci_status rci_set_refinement(rci_grid* g, double tol, int32_t max_steps);

/* Reciprocal solve of Eq. 7: v = A^{-dag} w = conj(A^{-1} conj(w)) (A symmetric).
 * v_src_out: DEVICE complex128[n_src], v on the source row j_src over S, or NULL.
 * v_full_out: DEVICE complex128[nx*ny], v on the whole grid, or NULL.
 * For VIRTUAL_FOCUS the propagator is
 *   K(D) = (h/pi) int_0^{pi/h} exp(i q(k) d_rows) cos(k D) dk,
 *   cos q = 2 - cos(k h) - k0^2 h^2 eps_air / 2, q >= 0 or q = i alpha, alpha > 0,
 * the exact continuation of a row of upward waves in homogeneous air on the
 * infinite lattice, evaluated by composite Gauss-Legendre quadrature.
 * Errors: ESTATE (not factored), EINVAL (objective outside the grid). */
rci_status rci_solve_reciprocal(rci_grid* g, const rci_objective* obj, double* v_src_out,
                                double* v_full_out, rci_info* info);

/* Averaged figure of merit by reciprocity (Eq. 7): one reciprocal solve, then
 *   F = sum_{i,l in S} conj(v_i) W(x_i - x_l) v_l
 * with W(D) = int rho(theta) cos(theta) exp(i k_s sin(theta) D) dtheta, k_s = 2 pi sqrt(eps_sub)
 * (closed forms: cone (sin c / c) sinc(k_s D sin c); annulus
 * [sin th2 sinc(k_s D sin th2) - sin th1 sinc(k_s D sin th1)] / (th2 - th1)), in
 * FP64 accumulation.  No h factors (arbitrary units).  out: HOST double. */
rci_status rci_avg_intensity(rci_grid* g, const rci_objective* obj, const rci_light* light,
                             double* out, rci_info* info);

/* Averaged figure of merit and its gradient with respect to the pillar widths, by
 * the adjoint of Eq. 7 (Sec. 4.1: dF = 2 Re(v^dag W dv), and dv costs one more solve
 * with the same factorisation).  With z = A^{-1} conj(w), v = conj(z) on S, g = W v:
 *   mu = A^{-1} P_S^T g   (second refined solve; A = A^T),
 *   dF/dw_m = -2 Re sum_c mu_c z_c k0^2 s_x s_y d(eps_c)/d(w_m),
 * where, in the pillar rows, d(eps_c)/d(w_m) = (eps_pillar - eps_air)/(2h) for each
 * column holding an edge of pillar m (the raster's area fill is piecewise linear in
 * the width).  At a tie (edge exactly on a column boundary) the derivative for a
 * growing width is taken.  value: HOST double (the same number rci_avg_intensity
 * returns).  dF_dwidths: HOST float64[n_cells].  Either may be NULL.
 * Errors: as rci_avg_intensity; ENOCONV if either solve ends above the tolerance
 * (outputs still written). */
rci_status rci_avg_intensity_grad(rci_grid* g, const rci_objective* obj, const rci_light* light,
                                  double* value, double* dF_dwidths, rci_info* info);

/* Averaged figure of merit for correlated incoherent light (Eq. 5 with Eq. 3): the
 * angular amplitude correlation <a(theta_q) a*(theta_q')> = C[q][q'] on a quadrature
 * (theta_q, weight_q = Omega_q) gives the cross-correlation
 *   W = sum_{q,q'} Omega_q Omega_q' C[q][q'] b0(theta_q) b0(theta_q')^dag
 * (b0 the unit-power planewave currents of rci_solve_angles), and by Eq. 7
 *   F = v^dag W v = sum_{q,q'} Omega_q Omega_q' C[q][q'] alpha_q conj(alpha_q'),
 *   alpha_q = v^dag b0(theta_q),
 * one reciprocal solve, an nq-point angular transform of v and an nq x nq Hermitian form,
 * in FP64.  Uncorrelated light is C = diag(rho_q / Omega_q).
 * theta, weight: HOST float64[nq] (|theta| < pi/2); C: HOST complex128[nq][nq], row-major,
 * Hermitian; 1 <= nq <= 8192.  out: HOST double. */
rci_status rci_avg_intensity_correlated(rci_grid* g, const rci_objective* obj, const double* theta,
                                        const double* weight, int64_t nq, const double* C,
                                        double* out, rci_info* info);

/* F = v^dag W v (Eq. 7) for a general cross-correlation given as a dense Hermitian matrix
 * on the source plane: W DEVICE complex128[n_src][n_src], row-major (W[i][l] couples
 * x_i and x_l, i, l in S), owned by the caller; read once per call.  out: HOST double. */
rci_status rci_avg_intensity_dense(rci_grid* g, const rci_objective* obj, const double* W,
                                   double* out, rci_info* info);

/* Several outputs at once (averages over several spots or modes, Sec. 6): for each
 * objective o, F_o = v_o^dag W v_o with v_o = A^{-dag} w_o, the K reciprocal solves done
 * as one multi-right-hand-side solve (chunks of 256) on the factorisation.
 * objs: HOST rci_objective[K], 1 <= K <= 65536.  F_out: HOST float64[K] or NULL;
 * total: HOST double (sum over the outputs, the trace objective) or NULL. */
rci_status rci_avg_intensity_multi(rci_grid* g, const rci_objective* objs, int64_t K,
                                   const rci_light* light, double* F_out, double* total,
                                   rci_info* info);

/* Brute-force average of Eq. 6 on the same factorisation: for each angle theta_q
 * (measured in the substrate) the equivalent current b0 = sqrt(cos theta) exp(i k_s
 * sin(theta) x_i) on row j_src over S, u_q = A^{-1} b0, f_q = |w^dag u_q|^2, and
 *   avg = sum_q weight_q f_q.
 * theta, weight: HOST float64[nq] (weight = quadrature weight times rho).
 * fom_per_angle: HOST float64[nq] or NULL.  avg_out: HOST double or NULL. */
rci_status rci_solve_angles(rci_grid* g, const rci_objective* obj, const double* theta,
                            const double* weight, int64_t nq, double* fom_per_angle,
                            double* avg_out, rci_info* info);

/* Brute-force average with an nq-point Gauss-Legendre rule (Sec. 5.2) on the
 * light's support (nq/2 points per interval for an annulus; nq even), rule built
 * on the device.  Outputs as rci_solve_angles (HOST, may be NULL). */
rci_status rci_avg_bruteforce(rci_grid* g, const rci_objective* obj, const rci_light* light,
                              int64_t nq, double* fom_per_angle, double* avg_out, rci_info* info);

/* FP64 Toeplitz quadratic form on the device:
 *   out = sum_{i,l < n} conj(v_i) lags[|i - l|] v_l
 * v: DEVICE complex128[n]; lags: DEVICE float64[n]; out: HOST double.
 * stream: cudaStream_t or NULL.  Allocates and frees a small device scratch. */
rci_status rci_qform_toeplitz(const double* v, const double* lags, int64_t n, double* out,
                              void* stream);

/* Allocation-free variant of rci_qform_toeplitz (the paper has no counterpart; this is
 * a library service).  rci_qform_toeplitz allocates its scratch with cudaMalloc and
 * releases it with cudaFree, and cudaFree synchronises the whole device.  Callers that
 * hand all device memory to their own pool, or that keep several streams busy and must
 * not be stalled by a device-wide synchronisation, call this one instead: it allocates
 * nothing, does not synchronise, and writes the result to device memory in stream order.
 *   out = sum_{i,l < n} conj(v_i) lags[|i - l|] v_l
 * v: DEVICE complex128[n]; lags: DEVICE float64[n]; out: DEVICE double[1];
 * stream: cudaStream_t or NULL.  1 <= n <= RCI_QFORM_NOALLOC_MAX_N, else RCI_EINVAL.
 * Scratch: a fixed device array of 32896 doubles (257 KB) inside the library, held by
 * every device that loads the library until the process exits and shared by all calls
 * on that device: calls that overlap on the GPU (e.g. on two streams) race.  Each call
 * overwrites all the scratch it reads, so nothing needs clearing between calls.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture. */
#define RCI_QFORM_NOALLOC_MAX_N 32768
rci_status rci_qform_toeplitz_noalloc(const double* v, const double* lags, int64_t n,
                                      double* out, void* stream);

/* n-point Gauss-Legendre rule on [a, b] computed on the device (Newton on the
 * three-term recurrence).  nodes, weights: DEVICE float64[n], ascending nodes. */
rci_status rci_gauss_legendre(int64_t n, double a, double b, double* nodes, double* weights,
                              void* stream);

/* Copies of the assembled problem, for inspection.  DEVICE outputs:
 * eps: float64[nx*ny] ([i][j]);  y = A x: complex128[nx*ny] (FP64 stencil). */
rci_status rci_get_eps(rci_grid* g, double* eps_out);
rci_status rci_apply_operator(rci_grid* g, const double* x, double* y);

/* Device bytes a grid of this descriptor holds once created: every buffer a single
 * right-hand-side evaluation needs (operator, factor store, solve workspace), plus the
 * gradient's buffers when with_gradient != 0, each allocation rounded up to 256 bytes.
 * Computed on the host without touching the device.  bytes: HOST.
 * Errors: EINVAL (bad descriptor). */
rci_status rci_grid_footprint(const rci_grid_desc* desc, int with_gradient, size_t* bytes);

/* ---- serving (continuous admission of many evaluations on one GPU) ----
 * The paper's use of the method is many evaluations: inverse design (Sec. 5.1) over
 * many designs and angular distributions.  A server runs `slots` workers (a host thread
 * and a CUDA stream each) over one device-memory arena taken at creation, so requests of
 * different sizes overlap on the device and admission never calls cudaMalloc/cudaFree.
 * A request is admitted when a worker is free and its grid (rci_grid_footprint with the
 * gradient buffers) can be carved out of the arena, after evicting resident
 * factorisations that no request is using (least recently used first); otherwise it
 * waits at the head of the queue for running requests to release memory.  A free worker
 * may start one of the next `lookahead` queued requests that fits while the head does
 * not (a head passed over 16 times is no longer overtaken).  A request that does not fit
 * in the arena even when nothing else holds memory completes with RCI_ENOMEM.  Each
 * evaluation is the one of rci_avg_intensity / rci_avg_intensity_grad on a grid of its
 * own, so its result does not depend on what else is in flight. */
typedef struct rci_server rci_server;

typedef struct {
  int32_t device;
  int32_t slots;          /* concurrent evaluations, 1..64 */
  uint64_t arena_bytes;   /* device memory taken at creation; 0: 90 % of the free memory */
  uint64_t cache_bytes;   /* at most this much of the arena keeps keyed factorisations
                             resident for reuse; 0: none are kept */
  int32_t lookahead;      /* >= 0; 0: strict first-in first-out admission */
  int32_t reserved;
} rci_server_desc;

typedef struct {
  rci_grid_desc grid;     /* geometry and precision (grid.device is ignored: the server's) */
  const double* widths;   /* HOST float64[grid.n_cells], copied by rci_server_submit */
  rci_objective obj;      /* USER_ROW's w_row is copied by rci_server_submit */
  rci_light light;        /* USER_LAGS's lags are copied by rci_server_submit */
  int32_t want_grad;      /* != 0: also dF/dwidths (rci_avg_intensity_grad) */
  int32_t reserved;
  uint64_t design_key;    /* != 0: the factorised grid may stay resident, and a later request
                             with the same key, descriptor and widths reuses it */
  double* grad_out;       /* HOST float64[grid.n_cells] when want_grad; owned by the caller,
                             must stay valid until the request completes; written before it
                             completes */
} rci_request;

typedef struct {
  int32_t status;         /* rci_status of the evaluation (RCI_ENOMEM: never fits) */
  int32_t cache_hit;      /* 1: a resident factorisation was reused */
  double value;           /* the averaged intensity F */
  int32_t refine_iters;
  int32_t fp64_fallback;  /* 1: the FP32 factorisation could not resolve the design and the
                             evaluation finished on the FP64 fallback (rci_info.fallback) */
  double rel_residual;
  double t_submit_us;     /* server clock: microseconds since rci_server_create */
  double t_start_us;      /* admitted (grid ready) */
  double t_end_us;        /* result ready */
  uint64_t footprint;     /* device bytes of the request's grid */
  int32_t simt_refactor;  /* 1: the design was factored again on the FP32 SIMT pipe
                             (rci_info.simt_refactor) */
  int32_t reserved;
} rci_result;

/* Server counters.  admission_waits: times a free worker found no queued request it could
 * admit for lack of memory and slept until a request finished or arrived; bypasses: requests
 * started ahead of the queue's head by the look-ahead. */
typedef struct {
  uint64_t submitted, completed, failed, cache_hits, cache_evictions, admission_waits, bypasses;
  int32_t in_flight, queued, resident, reserved;
  uint64_t arena_bytes, arena_used, arena_peak, cache_bytes;
} rci_server_stats;

/* Start a server (allocates the arena, creates the streams and workers).
 * Errors: EINVAL (bad descriptor), ENOMEM (arena), ECUDA. */
rci_status rci_server_create(const rci_server_desc* desc, rci_server** out);
/* Queue a request; returns at once with a ticket (HOST).  Inputs are copied.
 * Errors: EINVAL (bad request), ESTATE (server stopping). */
rci_status rci_server_submit(rci_server* s, const rci_request* req, uint64_t* ticket);
/* Wait for a ticket's result (HOST), timeout_s < 0: no limit.  Each ticket's result is
 * delivered once.  Errors: EINVAL (unknown or collected ticket), ETIMEOUT. */
rci_status rci_server_wait(rci_server* s, uint64_t ticket, double timeout_s, rci_result* out);
/* Counters and memory use.  out: HOST. */
rci_status rci_server_stats_read(rci_server* s, rci_server_stats* out);
/* Finish every queued request, stop the workers, release all device memory. */
rci_status rci_server_destroy(rci_server* s);

/* ---- instrumentation (no counterpart in the paper; measurement support) ----
 * Kernel families timed by the profiler:
 *   0 level-0 tridiagonal factor and first Schur blocks, 1 block inversions,
 *   2 factorisation GEMMs, 3 forward/backward substitution, 4 FP64 stencil residual,
 *   5 quadratic form, 6 raster/assembly/right-hand sides, 7 gradient (W v product and
 *   width chain rule; its solve counts under 3 and 4). */
#define RCI_PROFILE_FAMILIES 8
typedef struct {
  double ms[RCI_PROFILE_FAMILIES];      /* device time (CUDA events on the grid's stream) */
  double flops[RCI_PROFILE_FAMILIES];   /* algorithmic flops of the timed work */
  double bytes[RCI_PROFILE_FAMILIES];   /* algorithmic bytes of the timed work */
  int64_t launches[RCI_PROFILE_FAMILIES];
} rci_profile;

/* on != 0: reset the totals and start bracketing kernel families with CUDA events
 * (adds about a microsecond per family per call); on == 0: stop. */
rci_status rci_profile_enable(rci_grid* g, int on);
/* Totals since the last enable.  out: HOST. */
rci_status rci_profile_read(rci_grid* g, rci_profile* out);
/* Kernels launched by this library in this process so far. */
uint64_t rci_kernel_launches(void);

/* Batched inversion of complex n x n blocks with partial pivoting (the block-inverse step of
 * the factorisation behind rci_factor, exposed for reuse and testing; Sec. 4.1's single
 * solve rests on it):  out[z] = src[z]^{-1},  z < batch.
 * src, out: DEVICE arrays of batch row-major n x n blocks, contiguous, interleaved complex --
 * complex64 for prec = RCI_FP32_REFINE, complex128 for RCI_FP64; must not overlap; src may
 * be overwritten for n > 160.  kernel: 0 the factorisation's choice, 1 the SIMT Gauss-Jordan
 * kernels, 2 the tensor-core Gauss-Jordan (FP32 and n <= 160 only: tcgen05 3xTF32 panel
 * updates on the block held in tensor memory).  Pivot: largest |re| + |im| among the rows
 * not yet used.  Synchronises `stream` (cudaStream_t or NULL) and allocates a 4-byte
 * status word.  Errors: EINVAL, ESINGULAR (a zero pivot; out is then undefined), ETIMEOUT. */
rci_status rci_block_inverse(const void* src, void* out, int64_t n, int64_t batch, int32_t prec,
                             int32_t kernel, void* stream);

/* Batched complex GEMM of the block factorisation (instrumentation and tests; Sec. 4.2
 * leaves the solver open, and every level >= 1 of block cyclic reduction is built from these
 * products):
 *   C[z] = alpha op(A[z]) op(B[z]) + beta C0[z],   z = 0 .. batch-1,
 * op = identity (ta / tb == 0) or transpose (no conjugation), A[z] op-shaped M x K, B[z]
 * K x N, C[z] M x N; real alpha, beta.  Row-major DEVICE arrays of complex64 (prec
 * RCI_FP32_REFINE) or complex128 (RCI_FP64), leading dimensions lda, ldb, ldc0, ldc and element
 * strides sA, sB, sC0, sC between batch members (in complex elements); C0 may be NULL
 * (beta ignored).  C may equal C0 (same element positions), no other overlap.
 * kernel: 0 = the factorisation's dispatch; 1 = tensor cores (3xTF32 tcgen05), operands
 * staged through registers into shared memory; 2 = tensor cores fed by TMA with the A
 * operand in tensor memory (needs 2 <= N <= 160 and even, 16-byte aligned A, B, C, C0, even
 * leading dimensions and, for batch > 1, even positive sA, sB); 3 = SIMT.  Kernels 1 and 2
 * are FP32 only; the SIMT kernel (3, and 0 where it dispatches there: FP64, or batches too
 * small to fill the GPU) has no form with both operands transposed.  Synchronises `stream` (cudaStream_t or NULL) and allocates a 4-byte status
 * word.  Errors: EINVAL (sizes, a kernel that does not apply), ETIMEOUT, ECUDA. */
rci_status rci_cgemm_batched(int64_t M, int64_t N, int64_t K, int32_t ta, int32_t tb,
                             double alpha, const void* A, int64_t lda, int64_t sA, const void* B,
                             int64_t ldb, int64_t sB, double beta, const void* C0, int64_t ldc0,
                             int64_t sC0, void* C, int64_t ldc, int64_t sC, int64_t batch,
                             int32_t prec, int32_t kernel, void* stream);

/* Failure detection: every wait of a tensor-core pipeline stage (operand buffers,
 * accumulators) spins at most `cycles` SM clock cycles; a wait that runs out ends its
 * kernel (no trap), which records a device status that the next rci_factor / rci_solve
 * returns as RCI_ETIMEOUT; the kernel still waits, at the default limit, for its own
 * tensor-core operations before it frees its tensor memory, so the context stays usable.
 * Process-wide, applies to launches that start after the call; cycles <= 0 restores the
 * default (4e9 cycles, about 2 s).  Returns the previous limit.  Meant for tests of the
 * timeout path: a limit of a few hundred cycles makes the first pipeline wait run out. */
int64_t rci_set_wait_limit(int64_t cycles);

/* Arithmetic peaks of a device, measured by small loops on every SM, each about 30 ms
 * timed with CUDA events (instrumentation; the roofline fractions of the solver's kernels
 * divide by these).  FP32 FFMA and FP64 DFMA chains; the legacy warp-level FP64 (DMMA,
 * mma.sync m8n8k4) and INT8 (IMMA, mma.sync m16n8k32 s8) tensor paths -- sm_103a's
 * tcgen05 tensor cores take no INT8 operands; tcgen05.mma 128 x 256 from shared memory
 * in TF32 and in BF16.  Rates in 1e12 operations per second (a multiply-add counts 2).
 * Runs on its own stream and synchronises it; allocates a few bytes of device memory.
 * Errors: ECUDA, ETIMEOUT (a tensor-core probe's bounded completion wait expired). */
typedef struct {
  double fp32_fma_tflops;
  double fp64_fma_tflops;
  double fp64_dmma_tflops;
  double int8_imma_tops;
  double tf32_tcgen05_tflops;
  double bf16_tcgen05_tflops;
  int32_t sm_count;
  int32_t reserved;
} rci_peaks;
rci_status rci_measure_peaks(int device, rci_peaks* out);

/* Static strings; never NULL. */
const char* rci_status_str(rci_status s);
const char* rci_last_error(const rci_grid* g);

#ifdef __cplusplus
}
#endif
#endif /* RCI_H */
