// Correlated incoherent light and general (dense) cross-correlations.
//
// Eq. 5 with an angular amplitude correlation <a(theta) a*(theta')> that is not diagonal:
// on a quadrature (theta_q, Omega_q) with C[q][q'] = <a(theta_q) a*(theta_q')>, the
// equivalent currents have the cross-correlation of Eq. 3,
//     W = sum_{q,q'} Omega_q Omega_q' C[q][q'] b0(theta_q) b0(theta_q')^dag ,
// and Eq. 7 gives F = v^dag W v = sum_{q,q'} Omega_q Omega_q' C[q][q'] alpha_q conj(alpha_q')
// with alpha_q = v^dag b0(theta_q): one reciprocal solve, an nq-point angular transform
// of v and an nq x nq Hermitian form.  A general W given as a dense Hermitian matrix on
// the source plane is a plain v^dag W v, streamed from HBM once.
#include "kernels.cuh"

namespace {

constexpr int AA_THREADS = 256;
constexpr int DQ_WARPS = 8;

// fixed-order tree sum of a block's values in shared memory (blockDim.x a power of two)
__device__ __forceinline__ double block_sum(double x, double* sh) {
  sh[threadIdx.x] = x;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// alpha_q = sum_t conj(v_t) sqrt(cos theta_q) exp(i k_s sin(theta_q) x_t),  x_t = (t + 1/2) h
__global__ void __launch_bounds__(AA_THREADS)
angular_amp_kernel(GridGeom g, const double2* __restrict__ v, const double* __restrict__ theta,
                   double2* __restrict__ alpha) {
  __shared__ double sh[AA_THREADS];
  const int q = blockIdx.x;
  const double th = theta[q];
  const double amp = sqrt(cos(th)), kx = g.k_sub * sin(th);
  double ar = 0.0, ai = 0.0;
  for (int t = threadIdx.x; t < g.n_src; t += AA_THREADS) {
    double s, c;
    sincos(kx * ((t + 0.5) * g.h), &s, &c);
    const double2 vt = v[t];
    // conj(v) * (c + i s)
    ar += vt.x * c + vt.y * s;
    ai += vt.x * s - vt.y * c;
  }
  ar = block_sum(ar, sh);
  ai = block_sum(ai, sh);
  if (threadIdx.x == 0) alpha[q] = mkc(amp * ar, amp * ai);
}

// F = Re sum_q alpha_q sum_q' Om_q Om_q' C[q][q'] conj(alpha_q')   (one block)
__global__ void __launch_bounds__(AA_THREADS)
corr_form_kernel(const double2* __restrict__ alpha, const double* __restrict__ om,
                 const double2* __restrict__ C, int nq, double* __restrict__ out) {
  __shared__ double sh[AA_THREADS];
  double acc = 0.0;
  for (int q = threadIdx.x; q < nq; q += AA_THREADS) {
    double rr = 0.0, ri = 0.0;
    const double2* Cq = C + (int64_t)q * nq;
    for (int p = 0; p < nq; ++p) {
      const double2 c = Cq[p], a = alpha[p];
      const double w = om[p];
      // C[q][p] * conj(alpha_p) * Om_p
      rr += w * (c.x * a.x + c.y * a.y);
      ri += w * (c.y * a.x - c.x * a.y);
    }
    const double2 aq = alpha[q];
    acc += om[q] * (aq.x * rr - aq.y * ri);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[0] = acc;
}

// part[i] = Re conj(v_i) sum_l W[i][l] v_l, one warp per row (coalesced row reads)
__global__ void __launch_bounds__(DQ_WARPS * 32)
dense_rows_kernel(const double2* __restrict__ v, const double2* __restrict__ W, int64_t n,
                  double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * DQ_WARPS + (threadIdx.x >> 5);
  if (i >= n) return;
  const double2* Wi = W + i * n;
  double sr = 0.0, si = 0.0;
  for (int64_t l = lane; l < n; l += 32) {
    const double2 w = Wi[l], x = v[l];
    sr += w.x * x.x - w.y * x.y;
    si += w.x * x.y + w.y * x.x;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, off);
    si += __shfl_xor_sync(0xffffffffu, si, off);
  }
  if (lane == 0) {
    const double2 vi = v[i];
    part[i] = vi.x * sr + vi.y * si;
  }
}

// out = sum of part[0..n) in a fixed order (one block)
__global__ void __launch_bounds__(AA_THREADS)
sum_fixed_kernel(const double* __restrict__ part, int64_t n, double* __restrict__ out) {
  __shared__ double sh[AA_THREADS];
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += AA_THREADS) acc += part[k];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[0] = acc;
}

// B[k * ldq + q] = b[k]  (k < N): one right-hand side into a column of the multi-RHS layout
__global__ void put_column_kernel(const double2* __restrict__ b, int64_t N, int ldq, int q,
                                  double2* __restrict__ B) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) B[k * ldq + q] = b[k];
}

// v[t] = conj(X[((npml + t) ny + j_src) ldq + q])
__global__ void gather_source_col_kernel(GridGeom g, const double2* __restrict__ X, int ldq, int q,
                                         double2* __restrict__ v) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.n_src) return;
  v[t] = conj(X[((int64_t)(g.npml + t) * g.ny + g.j_src) * ldq + q]);
}

}  // namespace

cudaError_t launch_correlated_form(const GridGeom& g, const double2* v, const double* theta,
                                   const double* om, const double2* C, int nq, double2* alpha,
                                   double* out, cudaStream_t s) {
  if (nq < 1) return cudaErrorInvalidValue;
  angular_amp_kernel<<<nq, AA_THREADS, 0, s>>>(g, v, theta, alpha); rci_note_launch();
  RCI_CUDA_TRY(cudaGetLastError());
  corr_form_kernel<<<1, AA_THREADS, 0, s>>>(alpha, om, C, nq, out); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_dense_form(const double2* v, const double2* W, int64_t n, double* part,
                              double* out, cudaStream_t s) {
  if (n < 1) return cudaErrorInvalidValue;
  dense_rows_kernel<<<(unsigned)ceil_div(n, DQ_WARPS), DQ_WARPS * 32, 0, s>>>(v, W, n, part); rci_note_launch();
  RCI_CUDA_TRY(cudaGetLastError());
  sum_fixed_kernel<<<1, AA_THREADS, 0, s>>>(part, n, out); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_put_column(const double2* b, int64_t N, int ldq, int q, double2* B,
                              cudaStream_t s) {
  put_column_kernel<<<(unsigned)ceil_div(N, 256), 256, 0, s>>>(b, N, ldq, q, B); rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gather_source_col(const GridGeom& g, const double2* X, int ldq, int q,
                                     double2* v, cudaStream_t s) {
  gather_source_col_kernel<<<(unsigned)ceil_div(g.n_src, 128), 128, 0, s>>>(g, X, ldq, q, v); rci_note_launch();
  return cudaGetLastError();
}
