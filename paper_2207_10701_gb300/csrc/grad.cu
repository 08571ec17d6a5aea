// Width gradient of the averaged intensity by the adjoint method (Sec. 4.1: the
// gradient of v^dag W v is 2 Re(v^dag W dv), and dv costs one more solve with A).
//
// With z = A^{-1} conj(w), v = conj(z) on the source plane and g = W v:
//   dF = 2 Re(g^T dz_S),  dz = -A^{-1} dA z,  A = A^T
//   => mu = A^{-1} P_S^T g (one more solve),  dF = -2 Re sum_c mu_c z_c dA_cc .
// Only the diagonal depends on the design: dA_cc = k0^2 s_x s_y d eps_c, and in the
// pillar rows d eps_c / d w_m = (eps_pillar - eps_air) / (2h) for each column that
// holds an edge of pillar m (the area fill is piecewise linear in the width).
//
// Kernels here: the Toeplitz product g = W v (FP64, fixed summation order) and the
// per-pillar chain rule.  The second solve is the ordinary refined BCR solve.
#include "kernels.cuh"

namespace {

constexpr int TM_ROWS = 128;   // output rows per block (one per thread)
constexpr int TM_COLS = 1024;  // columns of W per block

// part[chunk][i] = sum_{l in chunk} W_{|i-l|} v_l for the 128 rows of this block.
// The lags the block needs, W_{|d|} for d = i - l over the tile, form one window of
// TM_COLS + TM_ROWS - 1 values that is staged in shared memory with the v tile.
__global__ void __launch_bounds__(TM_ROWS)
toeplitz_mv_kernel(const double2* __restrict__ v, const double* __restrict__ lags, int64_t n,
                   double2* __restrict__ part) {
  __shared__ double2 sv[TM_COLS];
  __shared__ double sl[TM_COLS + TM_ROWS];
  const int64_t i0 = (int64_t)blockIdx.x * TM_ROWS;
  const int64_t l0 = (int64_t)blockIdx.y * TM_COLS;
  const int64_t base = i0 - l0 - (TM_COLS - 1);  // d of window slot 0
  for (int t = threadIdx.x; t < TM_COLS + TM_ROWS - 1; t += TM_ROWS) {
    int64_t d = base + t;
    int64_t ad = d < 0 ? -d : d;
    sl[t] = ad < n ? lags[ad] : 0.0;
  }
  for (int c = threadIdx.x; c < TM_COLS; c += TM_ROWS) {
    int64_t l = l0 + c;
    sv[c] = l < n ? v[l] : mkc(0.0, 0.0);
  }
  __syncthreads();
  const int r = threadIdx.x;
  double ax = 0.0, ay = 0.0;
#pragma unroll 8
  for (int c = 0; c < TM_COLS; ++c) {
    double wl = sl[r - c + TM_COLS - 1];
    ax = fma(wl, sv[c].x, ax);
    ay = fma(wl, sv[c].y, ay);
  }
  int64_t i = i0 + r;
  if (i < n) part[(int64_t)blockIdx.y * n + i] = mkc(ax, ay);
}

// out[i] = sum over chunks in increasing order
__global__ void toeplitz_sum_kernel(const double2* __restrict__ part, int64_t n, int nchunk,
                                    double2* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 acc = part[i];
  for (int c = 1; c < nchunk; ++c) acc = acc + part[(int64_t)c * n + i];
  out[i] = acc;
}

// Lower bound of column i's extent, as the raster computes it.
__device__ __forceinline__ double col_lo(const GridGeom& g, int i) {
  double xi = __dmul_rn(__dadd_rn((double)(i - g.npml), 0.5), g.h);
  return __dsub_rn(xi, g.h / 2.0);
}
__device__ __forceinline__ double col_hi(const GridGeom& g, int i) {
  double xi = __dmul_rn(__dadd_rn((double)(i - g.npml), 0.5), g.h);
  return __dadd_rn(xi, g.h / 2.0);
}

// sum over the pillar rows of column i of Re(mu kss z)
__device__ __forceinline__ double column_term(const GridGeom& g, int i, const double2* mu,
                                              const double2* z, const double2* kss) {
  double acc = 0.0;
  for (int j = g.j_p0; j < g.j_p1; ++j) {
    int64_t k = (int64_t)i * g.ny + j;
    acc += (mu[k] * z[k] * kss[k]).x;
  }
  return acc;
}

// One thread per pillar.  The right edge b counts in every column with lo <= b < hi,
// the left edge a in every column with lo < a <= hi (the derivative for a growing
// width); the candidates around floor(x / h) are tested with the raster's own bounds.
__global__ void width_grad_kernel(GridGeom g, const double* __restrict__ widths,
                                  const double2* __restrict__ mu, const double2* __restrict__ z,
                                  const double2* __restrict__ kss, double* __restrict__ out) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.n_cells) return;
  double p = __dmul_rn((double)g.cell_px, g.h);
  double c = __dmul_rn(__dadd_rn((double)m, 0.5), p);
  double wh = widths[m] / 2.0;
  double a = __dsub_rn(c, wh), b = __dadd_rn(c, wh);
  double acc = 0.0;
  int ib = g.npml + (int)floor(b / g.h);
  for (int i = ib - 2; i <= ib + 2; ++i)
    if (i >= 0 && i < g.nx && col_lo(g, i) <= b && b < col_hi(g, i)) acc += column_term(g, i, mu, z, kss);
  int ia = g.npml + (int)floor(a / g.h);
  for (int i = ia - 2; i <= ia + 2; ++i)
    if (i >= 0 && i < g.nx && col_lo(g, i) < a && a <= col_hi(g, i)) acc += column_term(g, i, mu, z, kss);
  // -2 Re(...) * (eps_p - eps_air) / (2h)
  out[m] = -acc * __dsub_rn(g.eps_pillar, g.eps_air) / g.h;
}

}  // namespace

int64_t toeplitz_mv_chunks(int64_t n) { return ceil_div(n, TM_COLS); }

cudaError_t launch_toeplitz_mv(const double2* v, const double* lags, int64_t n, double2* part,
                               double2* out, cudaStream_t s) {
  if (n <= 0) return cudaErrorInvalidValue;
  int64_t nchunk = toeplitz_mv_chunks(n);
  int64_t nrow = ceil_div(n, TM_ROWS);
  if (nchunk > 65535 || nrow > 0x7fffffffLL) return cudaErrorInvalidValue;
  dim3 grd((unsigned)nrow, (unsigned)nchunk);
  toeplitz_mv_kernel<<<grd, TM_ROWS, 0, s>>>(v, lags, n, part); rci_note_launch();
  RCI_CUDA_TRY(cudaGetLastError());
  toeplitz_sum_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(part, n, (int)nchunk, out); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_width_grad(const GridGeom& g, const double* widths, const double2* mu,
                              const double2* z, const double2* kss, double* out, cudaStream_t s) {
  width_grad_kernel<<<(unsigned)ceil_div(g.n_cells, 128), 128, 0, s>>>(g, widths, mu, z, kss, out); rci_note_launch();
  return cudaGetLastError();
}
