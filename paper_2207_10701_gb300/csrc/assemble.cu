// Permittivity raster, FDFD operator assembly and the FP64 stencil kernels.
//
// Operator (the library's reading of the "Maxwell operator A" of Sec. 4.1): scalar
// Helmholtz with stretched-coordinate PML, scaled by s_x s_y so that A = A^T,
//   A u|_{ij} = s_y^j/h^2 [ (u_{i+1,j}-u_{ij})/s_x^{i+1/2} - (u_{ij}-u_{i-1,j})/s_x^{i-1/2} ]
//             + s_x^i/h^2 [ (u_{i,j+1}-u_{ij})/s_y^{j+1/2} - (u_{ij}-u_{i,j-1})/s_y^{j-1/2} ]
//             + k0^2 eps_ij s_x^i s_y^j u_ij ,     u = 0 outside the grid,
// s(xi) = 1 + i sigma_max (xi/d)^m / k0 with xi the depth into the PML, d = npml h.
// Coefficient arrays (FP64, [i][j] with j fastest):
//   dg[i][j]  diagonal,   cx[i][j] coupling (i,j)-(i+1,j) (i < nx-1),
//   cy[i][j]  coupling (i,j)-(i,j+1) (j < ny-1, last entry of a column is 0).
#include "kernels.cuh"

namespace {

__device__ __forceinline__ double2 stretch(const GridGeom& g, double depth) {
  double d = g.npml * g.h;
  double xi = depth > 0.0 ? depth : 0.0;
  double sig = g.sigma_max * pow(xi / d, (double)g.pml_m);
  return mkc(1.0, sig / g.k0);
}

// s_x at node i (half = false) or at the half node x_{i-1/2} (half = true)
__device__ __forceinline__ double2 sx_at(const GridGeom& g, int i, bool half) {
  double x = half ? (double)(i - g.npml) * g.h : ((double)(i - g.npml) + 0.5) * g.h;
  double dep = fmax(fmax(-x, x - g.width), 0.0);
  return stretch(g, dep);
}
__device__ __forceinline__ double2 sy_at(const GridGeom& g, int j, bool half) {
  double y = half ? (double)j * g.h : ((double)j + 0.5) * g.h;
  double y0 = g.npml * g.h, y1 = (g.ny - g.npml) * g.h;
  double dep = fmax(fmax(y0 - y, y - y1), 0.0);
  return stretch(g, dep);
}

// Fill fraction of grid column i in the pillar rows; the operation order follows the
// plain definition (sum over the pillars touching the column of the overlap length,
// divided by h) with no fused multiply-adds, so the result is reproducible bit for bit.
// Widths outside (0, period) are flagged in *status (DEV_BADINPUT); every width is
// seen by the columns of its own cell.
__global__ void raster_kernel(GridGeom g, const double* __restrict__ widths,
                              double* __restrict__ eps, const double2* __restrict__ dg0,
                              const double2* __restrict__ kss, double2* __restrict__ dg,
                              int32_t* status) {
  int i = blockIdx.y;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nx || j >= g.ny) return;
  double v;
  if (j < g.j_p0) {
    v = g.eps_sub;
  } else if (j >= g.j_p1) {
    v = g.eps_air;
  } else {
    double p = __dmul_rn((double)g.cell_px, g.h);
    double xi = __dmul_rn(__dadd_rn((double)(i - g.npml), 0.5), g.h);
    double half = g.h / 2.0;
    double lo = __dsub_rn(xi, half), hi = __dadd_rn(xi, half);
    int m0 = (int)floor(lo / p) - 1;
    int m1 = (int)floor(hi / p) + 1;
    if (m0 < 0) m0 = 0;
    if (m1 > g.n_cells - 1) m1 = g.n_cells - 1;
    double acc = 0.0;
    for (int m = m0; m <= m1; ++m) {
      double c = __dmul_rn(__dadd_rn((double)m, 0.5), p);
      double wm = widths[m];
      if (j == g.j_p0 && !(wm > 0.0 && wm < p)) atomicCAS(status, DEV_OK, DEV_BADINPUT);
      double wh = wm / 2.0;
      double a = __dsub_rn(c, wh), b = __dadd_rn(c, wh);
      double ov = __dsub_rn(fmin(hi, b), fmax(lo, a));
      acc = __dadd_rn(acc, ov > 0.0 ? ov : 0.0);
    }
    double f = acc / g.h;
    v = __dadd_rn(g.eps_air, __dmul_rn(f, __dsub_rn(g.eps_pillar, g.eps_air)));
  }
  int64_t k = (int64_t)i * g.ny + j;
  eps[k] = v;
  // the only permittivity-dependent coefficient: dg = dg0 + k0^2 eps s_x s_y
  double2 ks = kss[k];
  double2 d0 = dg0[k];
  dg[k] = mkc(fma(v, ks.x, d0.x), fma(v, ks.y, d0.y));
}

// Design-independent part of the stencil, computed once per grid:
//   dg0 = -s_y/h^2 (1/s_x^{i+1/2} + 1/s_x^{i-1/2}) - s_x/h^2 (1/s_y^{j+1/2} + 1/s_y^{j-1/2}),
//   kss = k0^2 s_x^i s_y^j,  cx, cy the couplings.
// The stretches depend on one coordinate each, so they are tabulated first (s at the node
// and 1/s at the half node below it, per column and per row) and combined per point.
__global__ void pml_tables_kernel(GridGeom g, double2* __restrict__ tx, double2* __restrict__ ty) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= g.nx) {
    tx[2 * t] = t < g.nx ? sx_at(g, t, false) : mkc(0.0, 0.0);
    tx[2 * t + 1] = crecip(sx_at(g, t, true));
  }
  int u = t - (g.nx + 1);
  if (u >= 0 && u <= g.ny) {
    ty[2 * u] = u < g.ny ? sy_at(g, u, false) : mkc(0.0, 0.0);
    ty[2 * u + 1] = crecip(sy_at(g, u, true));
  }
}

__global__ void pml_coeff_kernel(GridGeom g, const double2* __restrict__ tx,
                                 const double2* __restrict__ ty, double2* __restrict__ dg0,
                                 double2* __restrict__ kss, double2* __restrict__ cx,
                                 double2* __restrict__ cy) {
  int i = blockIdx.y;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nx || j >= g.ny) return;
  double h2 = g.h * g.h;
  double2 sx = tx[2 * i], sy = ty[2 * j];
  double2 isxm = tx[2 * i + 1], isxp = tx[2 * i + 3];
  double2 isym = ty[2 * j + 1], isyp = ty[2 * j + 3];
  double2 SYh = (1.0 / h2) * sy, SXh = (1.0 / h2) * sx;
  int64_t k = (int64_t)i * g.ny + j;
  dg0[k] = -(SYh * (isxp + isxm)) - SXh * (isyp + isym);
  kss[k] = (g.k0 * g.k0) * (sx * sy);
  if (i < g.nx - 1) cx[k] = SYh * isxp;
  cy[k] = (j < g.ny - 1) ? SXh * isyp : mkc(0.0, 0.0);
}

// y = A x (nrhs columns, [i][j][q])
__global__ void apply_A_kernel(GridGeom g, const double2* __restrict__ dg,
                               const double2* __restrict__ cx, const double2* __restrict__ cy,
                               const double2* __restrict__ x, double2* __restrict__ y, int nrhs) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t N = (int64_t)g.nx * g.ny;
  if (t >= N * nrhs) return;
  int64_t k = t / nrhs;
  int i = (int)(k / g.ny), j = (int)(k - (int64_t)i * g.ny);
  double2 acc = dg[k] * x[t];
  if (i > 0) acc = cfma(cx[k - g.ny], x[t - (int64_t)g.ny * nrhs], acc);
  if (i < g.nx - 1) acc = cfma(cx[k], x[t + (int64_t)g.ny * nrhs], acc);
  if (j > 0) acc = cfma(cy[k - 1], x[t - nrhs], acc);
  if (j < g.ny - 1) acc = cfma(cy[k], x[t + nrhs], acc);
  y[t] = acc;
}

constexpr int RES_THREADS = 256;
constexpr int RES_BLOCKS = 1216;  // 8 blocks on each of the 152 SMs (grid-stride loop)

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Single right-hand side: r = b - A x and per-block partial sums of |r|^2, |b|^2, reduced
// in a fixed order (warp shuffles, then warps in order), so the norms are reproducible.
__global__ void __launch_bounds__(RES_THREADS)
residual1_kernel(GridGeom g, const double2* __restrict__ dg, const double2* __restrict__ cx,
                 const double2* __restrict__ cy, const double2* __restrict__ b,
                 const double2* __restrict__ x, double2* __restrict__ r,
                 double* __restrict__ part_r, double* __restrict__ part_b) {
  __shared__ double wr[RES_THREADS / 32], wb[RES_THREADS / 32];
  const int N = g.nx * g.ny;
  double sr = 0.0, sb = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    int i = k / g.ny, j = k - i * g.ny;
    double2 acc = dg[k] * x[k];
    if (i > 0) acc = cfma(cx[k - g.ny], x[k - g.ny], acc);
    if (i < g.nx - 1) acc = cfma(cx[k], x[k + g.ny], acc);
    if (j > 0) acc = cfma(cy[k - 1], x[k - 1], acc);
    if (j < g.ny - 1) acc = cfma(cy[k], x[k + 1], acc);
    double2 bb = b[k];
    double2 rr = bb - acc;
    r[k] = rr;
    sr = fma(rr.x, rr.x, fma(rr.y, rr.y, sr));
    sb = fma(bb.x, bb.x, fma(bb.y, bb.y, sb));
  }
  sr = warp_sum_d(sr);
  sb = warp_sum_d(sb);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    wr[warp] = sr;
    wb[warp] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < RES_THREADS / 32; ++w) {
      a += wr[w];
      c += wb[w];
    }
    part_r[blockIdx.x] = a;
    part_b[blockIdx.x] = c;
  }
}

// Several right-hand sides: r = b - A x, and per-block partials of |r|^2 and |b|^2 for
// each right-hand side (grid-stride over unknowns; one partial per (block, q)).  The
// partials are gathered with shared-memory atomics, so these norms (used for the
// stopping test and the reported residual) may differ in the last bits between runs;
// r itself is exact to the order of the stencil sum.
__global__ void __launch_bounds__(RES_THREADS)
residual_kernel(GridGeom g, const double2* __restrict__ dg, const double2* __restrict__ cx,
                const double2* __restrict__ cy, const double2* __restrict__ b,
                const double2* __restrict__ x, double2* __restrict__ r, int nrhs,
                double* __restrict__ part_r, double* __restrict__ part_b) {
  extern __shared__ double red[];  // [2][RES_THREADS/32][nrhs]
  const int nw = RES_THREADS / 32;
  int warp = threadIdx.x >> 5;
  int64_t N = (int64_t)g.nx * g.ny;
  int64_t total = N * nrhs;
  for (int s = threadIdx.x; s < 2 * nw * nrhs; s += blockDim.x) red[s] = 0.0;
  __syncthreads();
  // each thread walks elements t = start + stride*c; q = t % nrhs
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = t / nrhs;
    int q = (int)(t - k * nrhs);
    int i = (int)(k / g.ny), j = (int)(k - (int64_t)i * g.ny);
    double2 acc = dg[k] * x[t];
    if (i > 0) acc = cfma(cx[k - g.ny], x[t - (int64_t)g.ny * nrhs], acc);
    if (i < g.nx - 1) acc = cfma(cx[k], x[t + (int64_t)g.ny * nrhs], acc);
    if (j > 0) acc = cfma(cy[k - 1], x[t - nrhs], acc);
    if (j < g.ny - 1) acc = cfma(cy[k], x[t + nrhs], acc);
    double2 bb = b[t];
    double2 rr = bb - acc;
    r[t] = rr;
    atomicAdd(&red[(0 * nw + warp) * nrhs + q], rr.x * rr.x + rr.y * rr.y);
    atomicAdd(&red[(1 * nw + warp) * nrhs + q], bb.x * bb.x + bb.y * bb.y);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nrhs; q += blockDim.x) {
    double sr = 0.0, sb = 0.0;
    for (int w = 0; w < nw; ++w) {
      sr += red[(0 * nw + w) * nrhs + q];
      sb += red[(1 * nw + w) * nrhs + q];
    }
    part_r[(int64_t)blockIdx.x * nrhs + q] = sr;
    part_b[(int64_t)blockIdx.x * nrhs + q] = sb;
  }
}

// out[q] = sqrt(sum_b part_r[b][q]) / sqrt(sum_b part_b[b][q]); one block per q, fixed-order
// strided sums then a tree.
__global__ void __launch_bounds__(256)
ratio_norms_kernel(const double* __restrict__ part_r, const double* __restrict__ part_b, int nblk,
                   int nrhs, double* __restrict__ out) {
  __shared__ double sr[256], sb[256];
  const int q = blockIdx.x;
  double a = 0.0, c = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    a += part_r[(int64_t)b * nrhs + q];
    c += part_b[(int64_t)b * nrhs + q];
  }
  sr[threadIdx.x] = a;
  sb[threadIdx.x] = c;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[q] = sb[0] > 0.0 ? sqrt(sr[0]) / sqrt(sb[0]) : sqrt(sr[0]);
}

__global__ void add_f32_kernel(double2* __restrict__ x, const float2* __restrict__ d, int64_t n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    float2 v = d[t];
    double2 a = x[t];
    x[t] = mkc(a.x + (double)v.x, a.y + (double)v.y);
  }
}
__global__ void axpy64_kernel(double2* __restrict__ x, const double2* __restrict__ d, int64_t n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] = x[t] + d[t];
}
__global__ void to_f32_kernel(const double2* __restrict__ a, float2* __restrict__ o, int64_t n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) o[t] = make_float2((float)a[t].x, (float)a[t].y);
}
__global__ void to_f64_kernel(const float2* __restrict__ a, double2* __restrict__ o, int64_t n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) o[t] = make_double2((double)a[t].x, (double)a[t].y);
}
__global__ void check_finite_kernel(const double2* __restrict__ a, int64_t n, int32_t* status) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    double2 v = a[t];
    if (!isfinite(v.x) || !isfinite(v.y)) atomicCAS(status, DEV_OK, DEV_NONFINITE);
  }
}

}  // namespace

cudaError_t launch_raster_eps(const GridGeom& g, const double* widths, double* eps,
                              const double2* dg0, const double2* kss, double2* dg,
                              int32_t* status, cudaStream_t s) {
  dim3 blk(64), grd((unsigned)ceil_div(g.ny, 64), (unsigned)g.nx);
  raster_kernel<<<grd, blk, 0, s>>>(g, widths, eps, dg0, kss, dg, status); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_pml_coefficients(const GridGeom& g, double2* dg0, double2* kss, double2* cx,
                                    double2* cy, double2* scratch, cudaStream_t s) {
  double2* tx = scratch;                      // 2 (nx + 1) entries
  double2* ty = scratch + 2 * (g.nx + 1);     // 2 (ny + 1) entries
  const int nt = g.nx + g.ny + 2;
  pml_tables_kernel<<<(unsigned)ceil_div(nt, 256), 256, 0, s>>>(g, tx, ty); rci_note_launch();
  RCI_CUDA_TRY(cudaGetLastError());
  dim3 blk(128), grd((unsigned)ceil_div(g.ny, 128), (unsigned)g.nx);
  pml_coeff_kernel<<<grd, blk, 0, s>>>(g, tx, ty, dg0, kss, cx, cy); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_apply_A(const GridGeom& g, const double2* dg, const double2* cx,
                           const double2* cy, const double2* x, double2* y, int nrhs,
                           cudaStream_t s) {
  int64_t total = (int64_t)g.nx * g.ny * nrhs;
  apply_A_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(g, dg, cx, cy, x, y, nrhs); rci_note_launch();
  return cudaGetLastError();
}

int residual_blocks(const GridGeom& g) {
  (void)g;
  return RES_BLOCKS;
}

cudaError_t launch_residual(const GridGeom& g, const double2* dg, const double2* cx,
                            const double2* cy, const double2* b, const double2* x, double2* r,
                            int nrhs, double* part_r, double* part_b, cudaStream_t s) {
  if (nrhs == 1) {
    residual1_kernel<<<RES_BLOCKS, RES_THREADS, 0, s>>>(g, dg, cx, cy, b, x, r, part_r, part_b);
    rci_note_launch();
    return cudaGetLastError();
  }
  size_t smem = sizeof(double) * 2 * (RES_THREADS / 32) * (size_t)nrhs;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024)
    RCI_CUDA_TRY(cudaFuncSetAttribute(residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  residual_kernel<<<RES_BLOCKS, RES_THREADS, smem, s>>>(g, dg, cx, cy, b, x, r, nrhs, part_r,
                                                        part_b); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ratio_norms(const double* part_r, const double* part_b, int nblk, int nrhs,
                               double* out, cudaStream_t s) {
  ratio_norms_kernel<<<(unsigned)nrhs, 256, 0, s>>>(part_r, part_b, nblk, nrhs, out);
  rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_add_f32(double2* x, const float2* d, int64_t n, cudaStream_t s) {
  add_f32_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(x, d, n); rci_note_launch();
  return cudaGetLastError();
}
cudaError_t launch_axpy64(double2* x, const double2* d, int64_t n, cudaStream_t s) {
  axpy64_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(x, d, n); rci_note_launch();
  return cudaGetLastError();
}
cudaError_t launch_to_f32(const double2* a, float2* o, int64_t n, cudaStream_t s) {
  to_f32_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(a, o, n); rci_note_launch();
  return cudaGetLastError();
}
cudaError_t launch_to_f64(const float2* a, double2* o, int64_t n, cudaStream_t s) {
  to_f64_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(a, o, n); rci_note_launch();
  return cudaGetLastError();
}
cudaError_t launch_check_finite(const double2* a, int64_t n, int32_t* status, cudaStream_t s) {
  check_finite_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(a, n, status); rci_note_launch();
  return cudaGetLastError();
}
