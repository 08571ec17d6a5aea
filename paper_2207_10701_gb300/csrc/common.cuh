// Shared device helpers: complex arithmetic on float2/double2, status word, launch checks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rci.h"

// ---------------------------------------------------------------- complex types
template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

__host__ __device__ __forceinline__ float2 mkc(float r, float i) { return make_float2(r, i); }
__host__ __device__ __forceinline__ double2 mkc(double r, double i) { return make_double2(r, i); }

template <typename T> __host__ __device__ __forceinline__ cplx<T> czero() { return mkc(T(0), T(0)); }

#define RCI_CPLX_OPS(V, S)                                                                      \
  __host__ __device__ __forceinline__ V operator+(V a, V b) { return mkc(a.x + b.x, a.y + b.y); } \
  __host__ __device__ __forceinline__ V operator-(V a, V b) { return mkc(a.x - b.x, a.y - b.y); } \
  __host__ __device__ __forceinline__ V operator-(V a) { return mkc(-a.x, -a.y); }               \
  __host__ __device__ __forceinline__ V operator*(V a, V b) {                                    \
    return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);                                    \
  }                                                                                              \
  __host__ __device__ __forceinline__ V operator*(S s, V a) { return mkc(s * a.x, s * a.y); }    \
  __host__ __device__ __forceinline__ V cfma(V a, V b, V acc) { /* acc + a*b */                  \
    acc.x = fma(a.x, b.x, acc.x);                                                                \
    acc.x = fma(-a.y, b.y, acc.x);                                                               \
    acc.y = fma(a.x, b.y, acc.y);                                                                \
    acc.y = fma(a.y, b.x, acc.y);                                                                \
    return acc;                                                                                  \
  }                                                                                              \
  __host__ __device__ __forceinline__ V cfms(V a, V b, V acc) { /* acc - a*b */                  \
    acc.x = fma(-a.x, b.x, acc.x);                                                               \
    acc.x = fma(a.y, b.y, acc.x);                                                                \
    acc.y = fma(-a.x, b.y, acc.y);                                                               \
    acc.y = fma(-a.y, b.x, acc.y);                                                               \
    return acc;                                                                                  \
  }                                                                                              \
  __host__ __device__ __forceinline__ V conj(V a) { return mkc(a.x, -a.y); }                     \
  __host__ __device__ __forceinline__ S cabs1(V a) { return fabs(a.x) + fabs(a.y); }             \
  __host__ __device__ __forceinline__ V crecip(V a) { /* 1/a, scaled to avoid overflow */        \
    S s = fabs(a.x) > fabs(a.y) ? fabs(a.x) : fabs(a.y);                                         \
    if (s == S(0)) return mkc(S(0), S(0));                                                       \
    S ar = a.x / s, ai = a.y / s;                                                                \
    S d = (ar * ar + ai * ai) * s;                                                               \
    return mkc(ar / d, -ai / d);                                                                 \
  }

RCI_CPLX_OPS(float2, float)
RCI_CPLX_OPS(double2, double)
#undef RCI_CPLX_OPS

template <typename To, typename From>
__host__ __device__ __forceinline__ cplx<To> ccast(From v) {
  return mkc(To(v.x), To(v.y));
}

// ---------------------------------------------------------------- device status word
// Kernels never trap.  They record the first failure here and the host reads it.
enum : int32_t { DEV_OK = 0, DEV_SINGULAR = 1, DEV_NONFINITE = 2, DEV_BADINPUT = 3, DEV_TIMEOUT = 4 };

// ---------------------------------------------------------------- launch helpers
#define RCI_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return _e;                       \
  } while (0)

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- device memory source
// Where a grid and its factorisation get their device memory: cudaMalloc / cudaFree by
// default, or an allocator supplied by the caller (the serving runtime's arena, whose
// allocations and releases never synchronise the device).
struct DevMem {
  void* ctx = nullptr;
  cudaError_t (*alloc_fn)(void* ctx, void** p, size_t bytes) = nullptr;
  void (*free_fn)(void* ctx, void* p) = nullptr;
  cudaError_t alloc(void** p, size_t bytes) const {
    if (bytes < 16) bytes = 16;
    return alloc_fn ? alloc_fn(ctx, p, bytes) : cudaMalloc(p, bytes);
  }
  void release(void* p) const {
    if (!p) return;
    if (free_fn)
      free_fn(ctx, p);
    else
      cudaFree(p);
  }
};

// ---------------------------------------------------------------- instrumentation
// Process-wide count of kernel launches made by this library (every launch site calls
// rci_note_launch), and an optional per-grid profiler that brackets kernel families
// with CUDA events on the launching stream and accumulates their device time together
// with the algorithmic flops / bytes of the work they did.
void rci_note_launch(int n = 1);

enum ProfFamily : int {
  PF_LEVEL0 = 0,   // tridiagonal factor + first Schur blocks
  PF_INVERT = 1,   // batched Gauss-Jordan inversions
  PF_GEMM = 2,     // batched complex GEMMs of the factorisation
  PF_SOLVE = 3,    // forward / backward substitution (all levels)
  PF_RESIDUAL = 4, // FP64 stencil residual + norms
  PF_QFORM = 5,    // Toeplitz quadratic form
  PF_SETUP = 6,    // raster, assembly, right-hand sides, conversions
  PF_GRAD = 7,     // Toeplitz product W v and the width chain rule of the gradient
  PF_COUNT = 8
};

struct Profiler {
  bool on = false;
  cudaEvent_t* pool = nullptr;
  int cap = 0, used = 0;
  struct Rec {
    int fam, e0, e1;
    double flops, bytes;
    int launches;
  };
  Rec* recs = nullptr;
  int nrec = 0;
  double ms[PF_COUNT] = {}, flops[PF_COUNT] = {}, bytes[PF_COUNT] = {};
  int64_t launches[PF_COUNT] = {};
  // returns an event index (or -1 when off / out of events)
  int mark(cudaStream_t s) {
    if (!on || used >= cap) return -1;
    cudaEventRecord(pool[used], s);
    return used++;
  }
  void add(int fam, int e0, int e1, double fl, double by, int nl) {
    if (!on || e0 < 0 || e1 < 0 || nrec >= cap) return;
    recs[nrec++] = Rec{fam, e0, e1, fl, by, nl};
  }
  // after the stream is synchronised: fold the recorded pairs into the totals
  void collect() {
    for (int r = 0; r < nrec; ++r) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pool[recs[r].e0], pool[recs[r].e1]) == cudaSuccess) {
        ms[recs[r].fam] += t;
        flops[recs[r].fam] += recs[r].flops;
        bytes[recs[r].fam] += recs[r].bytes;
        launches[recs[r].fam] += recs[r].launches;
      }
    }
    nrec = 0;
    used = 0;
  }
  void reset() {
    for (int f = 0; f < PF_COUNT; ++f) ms[f] = flops[f] = bytes[f] = 0, launches[f] = 0;
    nrec = 0;
    used = 0;
  }
};

// RAII bracket: PROF_SCOPE(prof, family, stream, flops, bytes, launches)
struct ProfScope {
  Profiler* p;
  int fam, e0;
  cudaStream_t s;
  double fl, by;
  int nl;
  ProfScope(Profiler* p_, int f, cudaStream_t s_, double fl_, double by_, int nl_)
      : p(p_), fam(f), e0(p_ ? p_->mark(s_) : -1), s(s_), fl(fl_), by(by_), nl(nl_) {}
  ~ProfScope() {
    if (p && e0 >= 0) p->add(fam, e0, p->mark(s), fl, by, nl);
  }
};
