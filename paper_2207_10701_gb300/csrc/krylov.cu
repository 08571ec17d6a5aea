// FP64 complex vector kernels of the Krylov refinement (flexible GMRES preconditioned by the
// FP32 factorisation; see refined_solve in capi.cu): several inner products at once, a
// combination of several vectors and scaling.  Reductions are two-pass with a fixed block count, so results do
// not depend on scheduling.
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int KV_THREADS = 256;
constexpr int KV_MAXV = KV_MAX_VECTORS;  // vectors per multi-dot / combination call

// part[b][i] = sum over block b's elements of conj(V_i[e]) w[e]  (i < nv)
__global__ void __launch_bounds__(KV_THREADS)
cdot_multi_kernel(const double2* __restrict__ V, int64_t ldv, int nv,
                  const double2* __restrict__ w, int64_t n, double2* __restrict__ part) {
  __shared__ double2 red[KV_THREADS / 32][KV_MAXV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double2 acc[KV_MAXV];
#pragma unroll
  for (int i = 0; i < KV_MAXV; ++i) acc[i] = make_double2(0.0, 0.0);
  for (int64_t e = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * KV_THREADS) {
    const double2 x = w[e];
#pragma unroll
    for (int i = 0; i < KV_MAXV; ++i) {
      if (i < nv) {
        const double2 v = V[(int64_t)i * ldv + e];
        // conj(v) x
        acc[i].x = fma(v.x, x.x, fma(v.y, x.y, acc[i].x));
        acc[i].y = fma(v.x, x.y, fma(-v.y, x.x, acc[i].y));
      }
    }
  }
#pragma unroll
  for (int i = 0; i < KV_MAXV; ++i) {
    if (i >= nv) break;
    double2 a = acc[i];
    for (int o = 16; o > 0; o >>= 1) {
      a.x += __shfl_down_sync(0xffffffffu, a.x, o);
      a.y += __shfl_down_sync(0xffffffffu, a.y, o);
    }
    if (lane == 0) red[warp][i] = a;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double2 t = make_double2(0.0, 0.0);
    for (int w8 = 0; w8 < KV_THREADS / 32; ++w8) {
      t.x += red[w8][threadIdx.x].x;
      t.y += red[w8][threadIdx.x].y;
    }
    part[(int64_t)blockIdx.x * KV_MAXV + threadIdx.x] = t;
  }
}

// out[i] = sum over blocks of part[b][i]
__global__ void cdot_sum_kernel(const double2* __restrict__ part, int nblk, int nv,
                                double2* __restrict__ out) {
  const int i = threadIdx.x;
  if (i >= nv) return;
  double2 t = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) {
    t.x += part[(int64_t)b * KV_MAXV + i].x;
    t.y += part[(int64_t)b * KV_MAXV + i].y;
  }
  out[i] = t;
}

// w += sign * sum_i coef[i] V_i
__global__ void __launch_bounds__(KV_THREADS)
caxpy_multi_kernel(double2* __restrict__ w, const double2* __restrict__ V, int64_t ldv, int nv,
                   const double2* __restrict__ coef, double sign, int64_t n) {
  __shared__ double2 c[KV_MAXV];
  if (threadIdx.x < nv) c[threadIdx.x] = make_double2(sign * coef[threadIdx.x].x,
                                                      sign * coef[threadIdx.x].y);
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * KV_THREADS) {
    double2 a = w[e];
    for (int i = 0; i < nv; ++i) {
      const double2 v = V[(int64_t)i * ldv + e];
      a.x = fma(c[i].x, v.x, fma(-c[i].y, v.y, a.x));
      a.y = fma(c[i].x, v.y, fma(c[i].y, v.x, a.y));
    }
    w[e] = a;
  }
}

__global__ void cscale_kernel(double2* __restrict__ out, const double2* __restrict__ in, double f,
                              int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = in[e];
    out[e] = make_double2(f * v.x, f * v.y);
  }
}

unsigned grid_for(int64_t n) {
  const int64_t g = (n + KV_THREADS - 1) / KV_THREADS;
  return (unsigned)(g < KV_DOT_BLOCKS ? (g > 0 ? g : 1) : KV_DOT_BLOCKS);
}

}  // namespace

cudaError_t launch_cdot_multi(const double2* V, int64_t ldv, int nv, const double2* w, int64_t n,
                              double2* part, double2* out, cudaStream_t s) {
  if (nv < 1 || nv > KV_MAXV) return cudaErrorInvalidValue;
  const unsigned nb = grid_for(n);
  cdot_multi_kernel<<<nb, KV_THREADS, 0, s>>>(V, ldv, nv, w, n, part);
  cdot_sum_kernel<<<1, KV_MAXV, 0, s>>>(part, (int)nb, nv, out);
  rci_note_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_caxpy_multi(double2* w, const double2* V, int64_t ldv, int nv,
                               const double2* coef, double sign, int64_t n, cudaStream_t s) {
  if (nv < 1 || nv > KV_MAXV) return cudaErrorInvalidValue;
  caxpy_multi_kernel<<<grid_for(n), KV_THREADS, 0, s>>>(w, V, ldv, nv, coef, sign, n);
  rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cscale(double2* out, const double2* in, double f, int64_t n, cudaStream_t s) {
  cscale_kernel<<<grid_for(n), KV_THREADS, 0, s>>>(out, in, f, n);
  rci_note_launch();
  return cudaGetLastError();
}
