// Sources, objectives, quadrature rules and cross-correlation lags.
//
// * Equivalent current of a unit-power planewave at angle theta in the substrate
//   (Sec. 4.1, principle of equivalence): sqrt(cos theta) exp(i k_s sin(theta) x_i) on
//   the source row over the interior columns.
// * Objective vectors w (Sec. 4.1): a node (concentrator), a planewave mode on a
//   monitor row (collimator), or the virtual-focus propagator row.
// * Gauss-Legendre rules (Sec. 5.2) and W(m h) in closed form (Eq. 4 and the
//   annulus formula of Sec. 5.1, with the cos(theta) Jacobian of the unit-power
//   amplitude: W(D) = int rho cos(theta) exp(i k_s sin(theta) D) dtheta).
#include "kernels.cuh"

namespace {

// ----------------------------------------------------------------- Gauss-Legendre
// Node k (1-based) of the n-point rule: Newton's method on the three-term recurrence
// (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1}, from x0 = cos(pi (k - 1/4) / (n + 1/2)).
__global__ void gl_kernel(int n, double a, double b, double* __restrict__ nodes,
                          double* __restrict__ weights) {
  int k = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (k > n) return;
  double x = cos(M_PI * (k - 0.25) / (n + 0.5));
  double p0 = 1.0, p1 = x, dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    p0 = 1.0;
    p1 = x;
    for (int m = 1; m < n; ++m) {
      double p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
      p0 = p1;
      p1 = p2;
    }
    dp = n * (x * p1 - p0) / (x * x - 1.0);
    double dx = p1 / dp;
    x -= dx;
    if (fabs(dx) < 1e-16) break;
  }
  p0 = 1.0;
  p1 = x;
  for (int m = 1; m < n; ++m) {
    double p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
    p0 = p1;
    p1 = p2;
  }
  dp = n * (x * p1 - p0) / (x * x - 1.0);
  double w = 2.0 / ((1.0 - x * x) * dp * dp);
  if (n == 1) {
    x = 0.0;
    w = 2.0;
  }
  int pos = n - k;  // ascending order
  nodes[pos] = 0.5 * (b - a) * x + 0.5 * (a + b);
  weights[pos] = 0.5 * (b - a) * w;
}

// ----------------------------------------------------------------- light
__global__ void light_rule_scale(int kind, double c, double th1, double th2, int nq,
                                 double* __restrict__ theta, double* __restrict__ wrho) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  double rho = kind == RCI_LIGHT_CONE ? 1.0 / (2.0 * c) : 1.0 / (2.0 * (th2 - th1));
  wrho[q] *= rho;
  (void)theta;
}

__device__ __forceinline__ double sinc_d(double z) {
  if (fabs(z) > 1e-4) return sin(z) / z;
  double z2 = z * z;
  return 1.0 - z2 / 6.0 + z2 * z2 / 120.0;
}

__global__ void w_lags_kernel(int kind, double c, double th1, double th2, double k_s, double h,
                              int64_t n, double* __restrict__ lags) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double D = h * (double)m;
  double v;
  if (kind == RCI_LIGHT_CONE) {
    double sc = sin(c);
    v = (sc / c) * sinc_d(k_s * D * sc);
  } else {
    double s1 = sin(th1), s2 = sin(th2);
    v = (s2 * sinc_d(k_s * D * s2) - s1 * sinc_d(k_s * D * s1)) / (th2 - th1);
  }
  lags[m] = v;
}

// Tabulated density (rci_light TABULATED): nodes of the composite rule in u = sin(theta).
// Sub-panel p lies in segment seg[p].x (between theta[q] and theta[q+1]), and is sub-panel
// seg[p].y of seg[p].z equal parts of that segment in u; TAB_ORDER Gauss-Legendre points each.
//   node[j] = (u_j, 2 w_j rho(asin u_j)),  since cos(theta) d theta = du
__global__ void tab_nodes_kernel(const double* __restrict__ theta, const double* __restrict__ rho,
                                 const int4* __restrict__ seg, int P, const double* __restrict__ gx,
                                 const double* __restrict__ gw, double2* __restrict__ node) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P * TAB_ORDER) return;
  const int p = j / TAB_ORDER, o = j - p * TAB_ORDER;
  const int4 sg = seg[p];
  const int q = sg.x;
  const double ua = sin(theta[q]), ub = sin(theta[q + 1]);
  const double a = ua + (ub - ua) * (double)sg.y / (double)sg.z;
  const double b = ua + (ub - ua) * (double)(sg.y + 1) / (double)sg.z;
  const double half = 0.5 * (b - a), mid = 0.5 * (a + b);
  const double u = mid + half * gx[o];
  const double th = asin(u);
  const double r = rho[q] + (rho[q + 1] - rho[q]) * (th - theta[q]) / (theta[q + 1] - theta[q]);
  node[j] = make_double2(u, 2.0 * half * gw[o] * r);
}

// lags[m] = sum_j c_j cos(k_s u_j m h), nodes staged through shared memory
constexpr int TAB_TILE = 256;
__global__ void __launch_bounds__(TAB_TILE)
tab_lags_kernel(const double2* __restrict__ node, int J, double k_s, double h, int64_t n,
                double* __restrict__ lags) {
  __shared__ double2 sn[TAB_TILE];
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double kd = k_s * h * (double)m;
  double acc = 0.0;
  for (int j0 = 0; j0 < J; j0 += TAB_TILE) {
    if (j0 + (int)threadIdx.x < J) sn[threadIdx.x] = node[j0 + threadIdx.x];
    __syncthreads();
    const int jn = J - j0 < TAB_TILE ? J - j0 : TAB_TILE;
    for (int j = 0; j < jn; ++j) acc = fma(sn[j].y, cos(kd * sn[j].x), acc);
    __syncthreads();
  }
  if (m < n) lags[m] = acc;
}

// ----------------------------------------------------------------- objectives / sources
__global__ void planewave_row_kernel(GridGeom g, double theta_out, double2* __restrict__ crow) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.n_src) return;
  double x = ((double)t + 0.5) * g.h;  // x_i for i = npml + t
  double s, c;
  sincos(g.k0 * sin(theta_out) * x, &s, &c);
  crow[t] = mkc(c, -s);  // conj(w_i), w_i = exp(i k0 sin(theta_out) x_i)
}

// Virtual focus: tables of the composite Gauss-Legendre rule in t, with k = k_c -+ t^2
// on the propagating / evanescent side of the branch point k_c (where q = 0).
//   prop[n]  = (k_n, Re, Im of exp(i q(k_n) D) 2 t_n w_n)
//   evan[n]  = (k_n, exp(-alpha(k_n) D) 2 t_n w_n)
__global__ void vf_tables_kernel(GridGeom g, int D, const double* __restrict__ gx,
                                 const double* __restrict__ gw, double* __restrict__ tab) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= VF_NODES) return;
  double h = g.h, k0 = g.k0, ea = g.eps_air;
  double kc = acos(1.0 - k0 * k0 * h * h * ea / 2.0) / h;
  double kmax = M_PI / h;
  int pnl = n / VF_ORDER, o = n - pnl * VF_ORDER;
  // propagating side
  {
    double tmax = sqrt(kc);
    double a = tmax * pnl / VF_PANELS, b = tmax * (pnl + 1) / VF_PANELS;
    double mid = 0.5 * (a + b), half = 0.5 * (b - a);
    double t = mid + half * gx[o], wt = half * gw[o];
    double k = kc - t * t;
    double cq = 2.0 - cos(k * h) - k0 * k0 * h * h * ea / 2.0;
    cq = fmin(fmax(cq, -1.0), 1.0);
    double q = acos(cq);
    double s, c;
    sincos(q * D, &s, &c);
    double f = 2.0 * t * wt;
    tab[4 * n + 0] = k;
    tab[4 * n + 1] = c * f;
    tab[4 * n + 2] = s * f;
  }
  // evanescent side
  {
    double tmax = sqrt(kmax - kc);
    double a = tmax * pnl / VF_PANELS, b = tmax * (pnl + 1) / VF_PANELS;
    double mid = 0.5 * (a + b), half = 0.5 * (b - a);
    double t = mid + half * gx[o], wt = half * gw[o];
    double k = kc + t * t;
    double cq = 2.0 - cos(k * h) - k0 * k0 * h * h * ea / 2.0;
    double al = acosh(fmax(cq, 1.0));
    tab[4 * VF_NODES + 2 * n + 0] = k;
    tab[4 * VF_NODES + 2 * n + 1] = exp(-al * D) * 2.0 * t * wt;
  }
}

// crow[t] = conj(w_t) = K(x_f - x_t): one block per column, block reduction.
__global__ void __launch_bounds__(256)
vf_row_kernel(GridGeom g, double x_f, const double* __restrict__ tab, double2* __restrict__ crow) {
  __shared__ double sr[256], si[256];
  int t = blockIdx.x;
  double delta = x_f - ((double)t + 0.5) * g.h;
  double ar = 0.0, ai = 0.0;
  for (int n = threadIdx.x; n < VF_NODES; n += blockDim.x) {
    double cp = cos(tab[4 * n] * delta);
    ar = fma(cp, tab[4 * n + 1], ar);
    ai = fma(cp, tab[4 * n + 2], ai);
    double ce = cos(tab[4 * VF_NODES + 2 * n] * delta);
    ar = fma(ce, tab[4 * VF_NODES + 2 * n + 1], ar);
  }
  sr[threadIdx.x] = ar;
  si[threadIdx.x] = ai;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double f = g.h / M_PI;
    crow[t] = mkc(f * sr[0], f * si[0]);
  }
}

__global__ void scatter_row_kernel(GridGeom g, const double2* __restrict__ crow, int row,
                                   double2* __restrict__ b) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.n_src) return;
  b[(int64_t)(g.npml + t) * g.ny + row] = crow[t];
}

__global__ void sources_kernel(GridGeom g, const double* __restrict__ theta, int nq, int ldq,
                               double2* __restrict__ B) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  int t = blockIdx.y;
  if (q >= nq || t >= g.n_src) return;
  double th = theta[q];
  double x = ((double)t + 0.5) * g.h;
  double s, c;
  sincos(g.k_sub * sin(th) * x, &s, &c);
  double a = sqrt(cos(th));
  B[((int64_t)(g.npml + t) * g.ny + g.j_src) * ldq + q] = mkc(a * c, a * s);
}

// amp_q = sum_t crow[t] U[(npml+t), row, q]; f_q = |amp_q|^2.  One block per q.
__global__ void __launch_bounds__(256)
project_row_kernel(GridGeom g, const double2* __restrict__ crow, int row,
                   const double2* __restrict__ U, int ldq, double* __restrict__ f) {
  __shared__ double sr[256], si[256];
  int q = blockIdx.x;
  double ar = 0.0, ai = 0.0;
  for (int t = threadIdx.x; t < g.n_src; t += blockDim.x) {
    double2 u = U[((int64_t)(g.npml + t) * g.ny + row) * ldq + q];
    double2 p = crow[t] * u;
    ar += p.x;
    ai += p.y;
  }
  sr[threadIdx.x] = ar;
  si[threadIdx.x] = ai;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) f[q] = sr[0] * sr[0] + si[0] * si[0];
}

__global__ void project_point_kernel(GridGeom g, int i_f, int j_f, const double2* __restrict__ U,
                                     int nq, int ldq, double* __restrict__ f) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  double2 u = U[((int64_t)i_f * g.ny + j_f) * ldq + q];
  f[q] = u.x * u.x + u.y * u.y;
}

__global__ void gather_source_row_kernel(GridGeom g, const double2* __restrict__ z,
                                         double2* __restrict__ v) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.n_src) return;
  v[t] = conj(z[(int64_t)(g.npml + t) * g.ny + g.j_src]);
}

__global__ void conj_kernel(double2* __restrict__ a, int64_t n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) a[t].y = -a[t].y;
}

__global__ void __launch_bounds__(256)
weighted_sum_kernel(const double* __restrict__ w, const double* __restrict__ f, int nq,
                    double* __restrict__ out) {
  __shared__ double s[256];
  double a = 0.0;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) a = fma(w[q], f[q], a);
  s[threadIdx.x] = a;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

}  // namespace

cudaError_t launch_gauss_legendre(int n, double a, double b, double* nodes, double* weights,
                                  cudaStream_t s) {
  if (n < 1) return cudaErrorInvalidValue;
  gl_kernel<<<(unsigned)ceil_div(n, 128), 128, 0, s>>>(n, a, b, nodes, weights); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_light_rule(int kind, double c, double th1, double th2, int nq, double* theta,
                              double* wrho, cudaStream_t s) {
  if (kind == RCI_LIGHT_CONE) {
    RCI_CUDA_TRY(launch_gauss_legendre(nq, -c, c, theta, wrho, s));
  } else {
    int half = nq / 2;
    RCI_CUDA_TRY(launch_gauss_legendre(half, -th2, -th1, theta, wrho, s));
    RCI_CUDA_TRY(launch_gauss_legendre(half, th1, th2, theta + half, wrho + half, s));
  }
  light_rule_scale<<<(unsigned)ceil_div(nq, 128), 128, 0, s>>>(kind, c, th1, th2, nq, theta,
                                                                wrho); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_w_lags(int kind, double c, double th1, double th2, double k_s, double h,
                          int64_t n, double* lags, cudaStream_t s) {
  w_lags_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(kind, c, th1, th2, k_s, h, n, lags); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_w_lags_tabulated(const double* theta, const double* rho, const int4* seg, int P,
                                   double* glx, double* glw, double2* node, double k_s, double h,
                                   int64_t n, double* lags, cudaStream_t s) {
  if (P < 1) return cudaErrorInvalidValue;
  RCI_CUDA_TRY(launch_gauss_legendre(TAB_ORDER, -1.0, 1.0, glx, glw, s));
  const int J = P * TAB_ORDER;
  tab_nodes_kernel<<<(unsigned)ceil_div(J, 128), 128, 0, s>>>(theta, rho, seg, P, glx, glw, node);
  rci_note_launch();
  RCI_CUDA_TRY(cudaGetLastError());
  tab_lags_kernel<<<(unsigned)ceil_div(n, TAB_TILE), TAB_TILE, 0, s>>>(node, J, k_s, h, n, lags);
  rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_planewave_row(const GridGeom& g, double theta_out, double2* crow,
                                 cudaStream_t s) {
  planewave_row_kernel<<<(unsigned)ceil_div(g.n_src, 128), 128, 0, s>>>(g, theta_out, crow); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_virtual_focus_row(const GridGeom& g, double x_f, int d_rows, double2* crow,
                                     double* scratch, cudaStream_t s) {
  double* gx = scratch;              // VF_ORDER nodes
  double* gw = scratch + VF_ORDER;   // VF_ORDER weights
  double* tab = scratch + 2 * VF_ORDER;  // 4*VF_NODES + 2*VF_NODES
  RCI_CUDA_TRY(launch_gauss_legendre(VF_ORDER, -1.0, 1.0, gx, gw, s));
  vf_tables_kernel<<<(unsigned)ceil_div(VF_NODES, 128), 128, 0, s>>>(g, d_rows, gx, gw, tab); rci_note_launch();
  RCI_CUDA_TRY(cudaGetLastError());
  vf_row_kernel<<<(unsigned)g.n_src, 256, 0, s>>>(g, x_f, tab, crow); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scatter_row(const GridGeom& g, const double2* crow, int row, double2* b,
                               cudaStream_t s) {
  scatter_row_kernel<<<(unsigned)ceil_div(g.n_src, 128), 128, 0, s>>>(g, crow, row, b); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sources(const GridGeom& g, const double* theta, int nq, int ldq, double2* B,
                           cudaStream_t s) {
  dim3 grd((unsigned)ceil_div(nq, 128), (unsigned)g.n_src);
  sources_kernel<<<grd, 128, 0, s>>>(g, theta, nq, ldq, B); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_project_row(const GridGeom& g, const double2* crow, int row,
                               const double2* U, int nq, int ldq, double* f, cudaStream_t s) {
  project_row_kernel<<<(unsigned)nq, 256, 0, s>>>(g, crow, row, U, ldq, f); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_project_point(const GridGeom& g, int i_f, int j_f, const double2* U, int nq,
                                 int ldq, double* f, cudaStream_t s) {
  project_point_kernel<<<(unsigned)ceil_div(nq, 128), 128, 0, s>>>(g, i_f, j_f, U, nq, ldq, f); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gather_source_row(const GridGeom& g, const double2* z, double2* v,
                                     cudaStream_t s) {
  gather_source_row_kernel<<<(unsigned)ceil_div(g.n_src, 128), 128, 0, s>>>(g, z, v); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_conj(double2* a, int64_t n, cudaStream_t s) {
  conj_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(a, n); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_weighted_sum(const double* w, const double* f, int nq, double* out,
                                cudaStream_t s) {
  weighted_sum_kernel<<<1, 256, 0, s>>>(w, f, nq, out); rci_note_launch();
  return cudaGetLastError();
}
