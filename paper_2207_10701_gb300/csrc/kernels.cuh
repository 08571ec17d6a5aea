// Host-side launchers of every kernel in the library (internal interface).
#pragma once

#include "common.cuh"

// ------------------------------------------------------------------ geometry
struct GridGeom {
  int nx, ny, npml, n_src, j_src, j_p0, j_p1, n_cells, cell_px;
  double h, k0, k_sub, eps_pillar, eps_sub, eps_air, sigma_max, width;
  int pml_m;
};

// assemble.cu
// per design: eps raster and the diagonal dg = dg0 + eps * kss (widths checked -> *status)
cudaError_t launch_raster_eps(const GridGeom& g, const double* widths_dev, double* eps,
                              const double2* dg0, const double2* kss, double2* dg,
                              int32_t* status, cudaStream_t s);
// once per grid: design-independent stencil parts (PML stretch, couplings); scratch holds
// at least 2 (nx + ny + 2) complex entries
cudaError_t launch_pml_coefficients(const GridGeom& g, double2* dg0, double2* kss, double2* cx,
                                    double2* cy, double2* scratch, cudaStream_t s);
cudaError_t launch_apply_A(const GridGeom& g, const double2* dg, const double2* cx,
                           const double2* cy, const double2* x, double2* y, int nrhs,
                           cudaStream_t s);
// r = b - A x and per-RHS partial sums of |r|^2 and |b|^2 (nblk x nrhs each)
int residual_blocks(const GridGeom& g);
cudaError_t launch_residual(const GridGeom& g, const double2* dg, const double2* cx,
                            const double2* cy, const double2* b, const double2* x, double2* r,
                            int nrhs, double* part_r, double* part_b, cudaStream_t s);
// sums the (nblk x nrhs) partials per column: out[q] = sqrt(sum r) / sqrt(sum b)
cudaError_t launch_ratio_norms(const double* part_r, const double* part_b, int nblk, int nrhs,
                               double* out, cudaStream_t s);
// x64 += (double) d (elementwise, n complex), optionally writes the float copy of r
cudaError_t launch_add_f32(double2* x, const float2* d, int64_t n, cudaStream_t s);
cudaError_t launch_to_f32(const double2* a, float2* out, int64_t n, cudaStream_t s);
cudaError_t launch_to_f64(const float2* a, double2* out, int64_t n, cudaStream_t s);
cudaError_t launch_axpy64(double2* x, const double2* d, int64_t n, cudaStream_t s);
cudaError_t launch_check_finite(const double2* a, int64_t n, int32_t* status, cudaStream_t s);

// krylov.cu: FP64 complex vectors of n elements, nv <= KV_MAX_VECTORS vectors V_i at V + i ldv.
constexpr int KV_MAX_VECTORS = 20;
constexpr int KV_DOT_BLOCKS = 4 * 152;  // blocks of the multi-dot (part holds
                                        // KV_DOT_BLOCKS x KV_MAX_VECTORS entries)
// out[i] = sum_e conj(V_i[e]) w[e]  (device out[nv]; part: device scratch)
cudaError_t launch_cdot_multi(const double2* V, int64_t ldv, int nv, const double2* w, int64_t n,
                              double2* part, double2* out, cudaStream_t s);
// w += sign sum_i coef[i] V_i  (coef: device, nv entries)
cudaError_t launch_caxpy_multi(double2* w, const double2* V, int64_t ldv, int nv,
                               const double2* coef, double sign, int64_t n, cudaStream_t s);
// out = f in (out may be in)
cudaError_t launch_cscale(double2* out, const double2* in, double f, int64_t n, cudaStream_t s);

// rhs.cu
cudaError_t launch_gauss_legendre(int n, double a, double b, double* nodes, double* weights,
                                  cudaStream_t s);
// conj(w) on the monitor row (n_src entries) for PLANEWAVE / VIRTUAL_FOCUS
cudaError_t launch_planewave_row(const GridGeom& g, double theta_out, double2* crow,
                                 cudaStream_t s);
cudaError_t launch_virtual_focus_row(const GridGeom& g, double x_f, int d_rows, double2* crow,
                                     double* scratch /* >= 2*VF_ORDER + 6*VF_NODES doubles */, cudaStream_t s);
constexpr int VF_PANELS = 256, VF_ORDER = 32, VF_NODES = VF_PANELS * VF_ORDER;
// scatter a row vector into a zeroed full-grid vector: b[(npml+t)*ny + row] = crow[t] (conj if asked)
cudaError_t launch_scatter_row(const GridGeom& g, const double2* crow, int row, double2* b,
                               cudaStream_t s);
// planewave sources for nq angles, [i][j][q] layout, into a zeroed buffer
cudaError_t launch_sources(const GridGeom& g, const double* theta, int nq, int ldq, double2* B,
                           cudaStream_t s);
// amp_q = sum_t crow[t] u[(npml+t)*ny + row][q]   (crow = conj(w));  f_q = |amp_q|^2
cudaError_t launch_project_row(const GridGeom& g, const double2* crow, int row,
                               const double2* U, int nq, int ldq, double* f, cudaStream_t s);
cudaError_t launch_project_point(const GridGeom& g, int i_f, int j_f, const double2* U, int nq,
                                 int ldq, double* f, cudaStream_t s);
// v_src[t] = conj(z[(npml+t)*ny + j_src])
cudaError_t launch_gather_source_row(const GridGeom& g, const double2* z, double2* v,
                                     cudaStream_t s);
cudaError_t launch_conj(double2* a, int64_t n, cudaStream_t s);
// light: rule (theta, weight*rho) for cone / annulus with nq points
cudaError_t launch_light_rule(int kind, double c, double th1, double th2, int nq, double* theta,
                              double* wrho, cudaStream_t s);
// W lags (closed forms) m = 0..n-1
// tabulated density: the composite rule's nodes (P sub-panels of TAB_ORDER points) and the
// lags; glx, glw: TAB_ORDER doubles each, node: P * TAB_ORDER entries (device scratch)
constexpr int TAB_ORDER = 12;
cudaError_t launch_w_lags_tabulated(const double* theta, const double* rho, const int4* seg, int P,
                                   double* glx, double* glw, double2* node, double k_s, double h,
                                   int64_t n, double* lags, cudaStream_t s);
cudaError_t launch_w_lags(int kind, double c, double th1, double th2, double k_s, double h,
                          int64_t n, double* lags, cudaStream_t s);
// weighted sum out = sum_q w_q f_q (single block, deterministic)
cudaError_t launch_weighted_sum(const double* w, const double* f, int nq, double* out,
                                cudaStream_t s);

// grad.cu
// g = W v for the real symmetric Toeplitz W (lags[0..n-1]); part holds
// toeplitz_mv_chunks(n) * n complex partials
int64_t toeplitz_mv_chunks(int64_t n);
cudaError_t launch_toeplitz_mv(const double2* v, const double* lags, int64_t n, double2* part,
                               double2* out, cudaStream_t s);
// out[m] = dF/dw_m = -2 Re sum_c mu_c z_c kss_c d eps_c/d w_m (pillar rows, edge columns)
cudaError_t launch_width_grad(const GridGeom& g, const double* widths, const double2* mu,
                              const double2* z, const double2* kss, double* out, cudaStream_t s);

// correlated.cu
// F = sum_{q,q'} om_q om_q' C[q][q'] alpha_q conj(alpha_q'), alpha_q = v^dag b0(theta_q)
cudaError_t launch_correlated_form(const GridGeom& g, const double2* v, const double* theta,
                                   const double* om, const double2* C, int nq, double2* alpha,
                                   double* out, cudaStream_t s);
// F = Re v^dag W v for a dense row-major W (n x n); part holds n doubles
cudaError_t launch_dense_form(const double2* v, const double2* W, int64_t n, double* part,
                              double* out, cudaStream_t s);
cudaError_t launch_put_column(const double2* b, int64_t N, int ldq, int q, double2* B,
                              cudaStream_t s);
cudaError_t launch_gather_source_col(const GridGeom& g, const double2* X, int ldq, int q,
                                     double2* v, cudaStream_t s);

// qform.cu
int64_t qform_num_partials(int64_t n);
cudaError_t launch_qform(const double2* v, const double* lags, int64_t n, double* partials,
                         double* out_dev, cudaStream_t s);
