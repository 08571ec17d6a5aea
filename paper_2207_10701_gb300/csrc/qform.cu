// Toeplitz quadratic form of Eq. 7 in FP64:
//   F = sum_{i,l < n} conj(v_i) W_{|i-l|} v_l ,  W real and even.
// Direct tiled reduction: the (i, l) plane is cut into 128 x 128 tiles; only tiles with
// tile_i >= tile_l are visited and off-diagonal tiles count twice (the form is real
// and the Toeplitz matrix symmetric).  Per pair two FP64 FMAs: the block accumulates
// s_i = sum_l W_{|i-l|} v_l, then adds Re(conj(v_i) s_i).  Per-tile partials are summed
// in a fixed order by a second kernel, so the result is bitwise reproducible.
#include <mutex>

#include "kernels.cuh"

namespace {

constexpr int QT = 128;

__device__ __forceinline__ void tile_of(int64_t b, int64_t& bi, int64_t& bl) {
  int64_t r = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while (r * (r + 1) / 2 > b) --r;
  while ((r + 1) * (r + 2) / 2 <= b) ++r;
  bi = r;
  bl = b - r * (r + 1) / 2;
}

__global__ void __launch_bounds__(QT)
qform_tile_kernel(const double2* __restrict__ v, const double* __restrict__ lags, int64_t n,
                  double* __restrict__ partials) {
  __shared__ double2 vl[QT];
  __shared__ double lw[2 * QT];
  __shared__ double red[QT];
  int64_t bi, bl;
  tile_of(blockIdx.x, bi, bl);
  int t = threadIdx.x;
  int64_t i = bi * QT + t;
  int64_t l0 = bl * QT;
  int64_t base = (bi - bl) * QT;  // i - l = base + (t - u)
  vl[t] = (l0 + t < n) ? v[l0 + t] : mkc(0.0, 0.0);
  for (int d = t; d < 2 * QT - 1; d += QT) {
    int64_t lag = base + d - (QT - 1);
    if (lag < 0) lag = -lag;
    lw[d] = lag < n ? lags[lag] : 0.0;
  }
  __syncthreads();
  double c = 0.0;
  if (i < n) {
    double sr = 0.0, si = 0.0;
#pragma unroll 8
    for (int u = 0; u < QT; ++u) {
      double wv = lw[t - u + QT - 1];
      double2 x = vl[u];
      sr = fma(wv, x.x, sr);
      si = fma(wv, x.y, si);
    }
    double2 vi = v[i];
    c = vi.x * sr + vi.y * si;
  }
  red[t] = c;
  __syncthreads();
  for (int s = QT / 2; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) partials[blockIdx.x] = (bi == bl ? 1.0 : 2.0) * red[0];
}

__global__ void __launch_bounds__(256)
sum_partials_kernel(const double* __restrict__ p, int64_t np, double* __restrict__ out) {
  __shared__ double s[256];
  double a = 0.0;
  for (int64_t k = threadIdx.x; k < np; k += blockDim.x) a += p[k];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

}  // namespace

int64_t qform_num_partials(int64_t n) {
  int64_t nb = ceil_div(n, QT);
  return nb * (nb + 1) / 2;
}

cudaError_t launch_qform(const double2* v, const double* lags, int64_t n, double* partials,
                         double* out_dev, cudaStream_t s) {
  if (n <= 0) return cudaErrorInvalidValue;
  int64_t np = qform_num_partials(n);
  if (np > 0x7fffffffLL) return cudaErrorInvalidValue;
  qform_tile_kernel<<<(unsigned)np, QT, 0, s>>>(v, lags, n, partials); rci_note_launch();
  RCI_CUDA_TRY(cudaGetLastError());
  sum_partials_kernel<<<1, 256, 0, s>>>(partials, np, out_dev); rci_note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- allocation-free variant
// rci_qform_toeplitz allocates its per-tile partials with cudaMalloc and releases them
// with cudaFree, which synchronises the whole device.  Callers that own all device
// memory through their own pool, or that overlap work on several streams and must not
// be stalled by a device-wide synchronisation, use rci_qform_toeplitz_noalloc instead:
// its partials live in the file-scope array below, which every device that loads this
// library holds until the process exits.
//
// The array is shared by every call on a device.  Each call writes every partial it
// later reads and then the result, so nothing has to start at zero and stale contents
// of an earlier (larger) call are never read; two calls that overlap on the GPU (for
// example on two streams) race on the array.
namespace {
constexpr int64_t NOALLOC_TILES = RCI_QFORM_NOALLOC_MAX_N / QT;                // 256
constexpr int64_t NOALLOC_PARTIALS = NOALLOC_TILES * (NOALLOC_TILES + 1) / 2;  // 32896
constexpr int NOALLOC_MAX_DEVICES = 64;
static_assert(RCI_QFORM_NOALLOC_MAX_N % QT == 0, "maximum size must be a whole number of tiles");
}  // namespace

static __device__ __align__(256) double g_qform_noalloc_scratch[NOALLOC_PARTIALS];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up with that device current
// and cached once found; a failed lookup is not cached, so a later call tries again.
cudaError_t noalloc_scratch(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_qform_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" rci_status rci_qform_toeplitz_noalloc(const double* v, const double* lags, int64_t n,
                                                 double* out, void* stream) {
  if (!v || !lags || !out || n < 1) return RCI_EINVAL;
  if (n > RCI_QFORM_NOALLOC_MAX_N) return RCI_EINVAL;
  double* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return RCI_ECUDA;
  if (launch_qform((const double2*)v, lags, n, scratch, out, (cudaStream_t)stream) != cudaSuccess)
    return RCI_ECUDA;
  return RCI_OK;
}
