// Arithmetic peaks of the device the library runs on, measured with small loops (no
// counterpart in the paper; the roofline fractions of the solver's kernels divide by these).
//
//   FP32 FFMA and FP64 DFMA     independent fused multiply-add chains on every SM
//   FP64 DMMA                   legacy warp-level mma.sync m8n8k4 (f64)
//   INT8 IMMA                   legacy warp-level mma.sync m16n8k32 (s8 x s8 -> s32); the
//                               5th-generation tensor cores take no INT8 operands on sm_103a
//                               (tcgen05.mma kind::i8 does not assemble for this target)
//   TF32 / BF16 tcgen05         one thread per SM issuing 128 x 256 x K tcgen05.mma from
//                               shared memory into two tensor-memory accumulators
//
// Each probe runs once briefly to calibrate, then for about 30 ms, timed with CUDA events
// on a private stream.  The one wait in these kernels (for the last tensor-core operation
// before tensor memory is freed) is bounded.
#include <cstring>

#include "common.cuh"

namespace {

constexpr int FMA_CHAINS = 8, FMA_UNROLL = 16, FMA_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(FMA_THREADS) fma_probe_kernel(T* sink, long long iters, T seed) {
  T a[FMA_CHAINS];
#pragma unroll
  for (int i = 0; i < FMA_CHAINS; ++i) a[i] = seed + T(0.01) * (T)(i + threadIdx.x % 7);
  const T b = T(0.999), c = T(0.001);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < FMA_UNROLL; ++r)
#pragma unroll
      for (int i = 0; i < FMA_CHAINS; ++i) a[i] = fma(a[i], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < FMA_CHAINS; ++i) s += a[i];
  if (s == T(-1)) sink[blockIdx.x] = s;  // never true; keeps the chains alive
}

constexpr int MMA_THREADS = 256, MMA_ACC = 4;

__global__ void __launch_bounds__(MMA_THREADS) dmma_probe_kernel(double* sink, long long iters) {
  double c[MMA_ACC][2];
  const double a = 1.0 + 1e-3 * (threadIdx.x & 31), b = 0.5;
#pragma unroll
  for (int k = 0; k < MMA_ACC; ++k) c[k][0] = c[k][1] = 0.0;
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < MMA_ACC; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < MMA_ACC; ++k) s += c[k][0] + c[k][1];
  if (s == -1.0) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(MMA_THREADS) imma_probe_kernel(int* sink, long long iters) {
  int c[MMA_ACC][4];
  const uint32_t a0 = 0x01020304u + threadIdx.x, b0 = 0x01010101u;
#pragma unroll
  for (int k = 0; k < MMA_ACC; ++k) c[k][0] = c[k][1] = c[k][2] = c[k][3] = 0;
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < MMA_ACC; ++k)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};"
          : "+r"(c[k][0]), "+r"(c[k][1]), "+r"(c[k][2]), "+r"(c[k][3])
          : "r"(a0), "r"(a0), "r"(a0), "r"(a0), "r"(b0), "r"(b0));
  }
  int s = 0;
#pragma unroll
  for (int k = 0; k < MMA_ACC; ++k) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
  if (s == -1) sink[blockIdx.x] = s;
}

// ---- tcgen05: M = 128, N = 256, operands K-major without swizzle (8-row x 16-byte core
// matrices; LBO = next core matrix along K, SBO = next 8-row group)
constexpr int TC_M = 128, TC_N = 256;
constexpr uint32_t TC_ROW_BYTES = 32;                 // one K block: 8 tf32 or 16 bf16 values
constexpr uint32_t TC_LBO = 128, TC_SBO = 256;
constexpr uint32_t TC_A_BYTES = TC_M * TC_ROW_BYTES;  // 4 KB
constexpr uint32_t TC_B_BYTES = TC_N * TC_ROW_BYTES;  // 8 KB
constexpr long long TC_WAIT_LIMIT = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t desc_of(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind: 0 = tf32 (A, B format 2), 1 = bf16 under kind::f16 (format 1); D = F32
// Launched with TC_PROBE_SMEM bytes of dynamic shared memory, more than half of an SM's,
// so that one CTA runs per SM and owns all 512 tensor-memory columns.
constexpr int TC_PROBE_SMEM = 120 * 1024;

template <int KIND>
__global__ void __launch_bounds__(128, 1) tcgen05_probe_kernel(long long iters, int32_t* status) {
  extern __shared__ __align__(1024) unsigned char ops[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  // operands: small non-zero values (the bit patterns are valid tf32 / bf16 numbers)
  for (uint32_t e = tid; e < (TC_A_BYTES + TC_B_BYTES) / 4; e += 128) {
    const uint32_t v = KIND == 0 ? (0x3F800000u ^ ((e * 2654435761u) & 0x007FE000u))
                                 : (0x3F803F80u ^ ((e * 2654435761u) & 0x007F007Fu));
    reinterpret_cast<uint32_t*>(ops)[e] = v;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    constexpr uint32_t fmt = KIND == 0 ? 2u : 1u;
    constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) |
                               ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    const uint64_t ad = desc_of(smem_u32(ops)), bd = desc_of(smem_u32(ops + TC_A_BYTES));
    for (long long it = 0; it < iters; ++it) {
      const uint32_t d = tmem + (uint32_t)(it & 1) * 256u;
      const uint32_t acc = it >= 2 ? 1u : 0u;
      if (KIND == 0)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&bar))
        : "memory");
    const long long t0 = clock64();
    while (true) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(&bar))
          : "memory");
      if (done) break;
      if (clock64() - t0 > TC_WAIT_LIMIT) {
        atomicCAS(status, DEV_OK, DEV_TIMEOUT);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

struct Probe {
  cudaStream_t s;
  cudaEvent_t e0, e1;
  void* sink;
  int32_t* status;
  int nsm;
};

// Runs launch(iters) once with iters0 to calibrate, then with the iteration count that
// takes about target_ms; returns operations per second from the second run.
template <typename F>
cudaError_t timed(Probe& p, long long iters0, double ops_per_iter, double target_ms, F launch,
                  double* ops_per_s) {
  float ms = 0.f;
  RCI_CUDA_TRY(launch(iters0));  // first touch (module load, clocks up)
  RCI_CUDA_TRY(cudaEventRecord(p.e0, p.s));
  RCI_CUDA_TRY(launch(iters0));
  RCI_CUDA_TRY(cudaEventRecord(p.e1, p.s));
  RCI_CUDA_TRY(cudaEventSynchronize(p.e1));
  RCI_CUDA_TRY(cudaEventElapsedTime(&ms, p.e0, p.e1));
  double scale = ms > 0.f ? target_ms / ms : 1.0;
  if (scale > 1e4) scale = 1e4;
  const long long iters = (long long)(iters0 * (scale < 1.0 ? 1.0 : scale)) + 1;
  RCI_CUDA_TRY(cudaEventRecord(p.e0, p.s));
  RCI_CUDA_TRY(launch(iters));
  RCI_CUDA_TRY(cudaEventRecord(p.e1, p.s));
  RCI_CUDA_TRY(cudaEventSynchronize(p.e1));
  RCI_CUDA_TRY(cudaEventElapsedTime(&ms, p.e0, p.e1));
  *ops_per_s = ms > 0.f ? ops_per_iter * (double)iters / (ms * 1e-3) : 0.0;
  return cudaSuccess;
}

cudaError_t measure(Probe& p, rci_peaks* out) {
  const int blocks = p.nsm * 8;  // 8 x 256 threads per SM: full occupancy for the FMA loops
  const double thr = (double)blocks * FMA_THREADS;
  const double fma_ops = 2.0 * FMA_CHAINS * FMA_UNROLL * thr;
  double v = 0.0;
  RCI_CUDA_TRY(timed(p, 64, fma_ops, 30.0, [&](long long it) {
    fma_probe_kernel<float><<<blocks, FMA_THREADS, 0, p.s>>>((float*)p.sink, it, 1.0f);
    rci_note_launch();
    return cudaGetLastError();
  }, &v));
  out->fp32_fma_tflops = v * 1e-12;
  RCI_CUDA_TRY(timed(p, 4, fma_ops, 30.0, [&](long long it) {
    fma_probe_kernel<double><<<blocks, FMA_THREADS, 0, p.s>>>((double*)p.sink, it, 1.0);
    rci_note_launch();
    return cudaGetLastError();
  }, &v));
  out->fp64_fma_tflops = v * 1e-12;
  const double warps = (double)blocks * (MMA_THREADS / 32);
  RCI_CUDA_TRY(timed(p, 4, warps * MMA_ACC * 2.0 * 8 * 8 * 4, 30.0, [&](long long it) {
    dmma_probe_kernel<<<blocks, MMA_THREADS, 0, p.s>>>((double*)p.sink, it);
    rci_note_launch();
    return cudaGetLastError();
  }, &v));
  out->fp64_dmma_tflops = v * 1e-12;
  RCI_CUDA_TRY(timed(p, 16, warps * MMA_ACC * 2.0 * 16 * 8 * 32, 30.0, [&](long long it) {
    imma_probe_kernel<<<blocks, MMA_THREADS, 0, p.s>>>((int*)p.sink, it);
    rci_note_launch();
    return cudaGetLastError();
  }, &v));
  out->int8_imma_tops = v * 1e-12;
  const double tf32_ops = (double)p.nsm * 2.0 * TC_M * TC_N * 8;
  RCI_CUDA_TRY(cudaFuncSetAttribute(tcgen05_probe_kernel<0>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, TC_PROBE_SMEM));
  RCI_CUDA_TRY(cudaFuncSetAttribute(tcgen05_probe_kernel<1>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, TC_PROBE_SMEM));
  RCI_CUDA_TRY(timed(p, 256, tf32_ops, 30.0, [&](long long it) {
    tcgen05_probe_kernel<0><<<p.nsm, 128, TC_PROBE_SMEM, p.s>>>(it, p.status);
    rci_note_launch();
    return cudaGetLastError();
  }, &v));
  out->tf32_tcgen05_tflops = v * 1e-12;
  RCI_CUDA_TRY(timed(p, 256, 2.0 * tf32_ops, 30.0, [&](long long it) {
    tcgen05_probe_kernel<1><<<p.nsm, 128, TC_PROBE_SMEM, p.s>>>(it, p.status);
    rci_note_launch();
    return cudaGetLastError();
  }, &v));
  out->bf16_tcgen05_tflops = v * 1e-12;
  return cudaSuccess;
}

}  // namespace

extern "C" rci_status rci_measure_peaks(int device, rci_peaks* out) {
  if (!out) return RCI_EINVAL;
  std::memset(out, 0, sizeof(*out));
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
    return RCI_ECUDA;
  Probe p{};
  cudaError_t e = cudaDeviceGetAttribute(&p.nsm, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p.s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&p.e0);
  if (e == cudaSuccess) e = cudaEventCreate(&p.e1);
  if (e == cudaSuccess) e = cudaMalloc(&p.sink, (size_t)p.nsm * 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p.status, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(p.status, 0, sizeof(int32_t), p.s);
  if (e == cudaSuccess) e = measure(p, out);
  int32_t st = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, p.status, sizeof(st), cudaMemcpyDeviceToHost, p.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p.s);
  out->sm_count = p.nsm;
  if (p.s) cudaStreamSynchronize(p.s);
  if (p.sink) cudaFree(p.sink);
  if (p.status) cudaFree(p.status);
  if (p.e0) cudaEventDestroy(p.e0);
  if (p.e1) cudaEventDestroy(p.e1);
  if (p.s) cudaStreamDestroy(p.s);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RCI_ENOMEM : RCI_ECUDA;
  return st == DEV_OK ? RCI_OK : RCI_ETIMEOUT;
}
