// Batched complex FP32 block inversion with partial pivoting on the 5th-generation tensor
// cores: blocked Gauss-Jordan whose rank-16 updates run as tcgen05.mma (3xTF32) on a copy
// of the block held in tensor memory.
//
// Algebra (the same as the SIMT look-ahead kernel in bcr.cu).  For each panel of 16
// columns K = [c0, c0 + 16):
//   1. 16 unblocked Gauss-Jordan steps restricted to the panel columns: the pivot of column
//      k is the unused row with the largest |re| + |im| (ties to the lowest row), recorded
//      as piv[k] instead of swapping rows; the pivot row is scaled, every other row is
//      eliminated, and the pivot column turns into -column / pivot with 1 / pivot on the
//      pivot row (the in-place inverse).
//   2. every column j outside the panel gets the product of the panel's elementary
//      transforms: with R[u][j] = M[piv[c0 + u]][j] (the pivot rows before the update),
//        M[i][j] <- (i a pivot row of the panel ? 0 : M[i][j]) + sum_u M[i][c0 + u] R[u][j].
//   The inverse is M[piv[i]][pinv[j]] with pinv the inverse permutation of piv.
//
// Layout.  The block (padded to np = a multiple of 16 with identity rows and columns) lives
// in tensor memory as the stacked real matrix [Re M; Im M] in 128-lane tiles: complex row
// r < 128 has its real part in lane r of tile 0 and its imaginary part in lane r of tile 1;
// rows 128 .. 159 sit in tile 2, real part in lane 32 g + t and imaginary part in lane
// 32 g + 16 + t for r = 128 + 16 g + t, so that both parts of a row are always read by the
// same warp (warp w reads lanes 32 w .. 32 w + 31).  Tile tau occupies tensor-memory
// columns [tau TS, tau TS + np), matrix column j at column tau TS + j.
//
// The update of step 2 is one real product per tile: the accumulator D (the tile, in
// tensor memory) += A B with A the panel in stacked form, row (r, Re) = (Re P[r][u],
// -Im P[r][u]) and row (r, Im) = (Im P[r][u], Re P[r][u]) over u, and B = (Re R[u][j],
// Im R[u][j]) over u, K = 32 real; each operand split into TF32 hi + lo, three MMAs
// (hi hi, hi lo, lo hi) per 8-deep K step, FP32 accumulation.  The pivot rows' zeroing is a
// read-modify-write of tensor memory that also collects R.
//
// Schedule of one block (one CTA of 4 warps per SM, persistent over the batch):
//   load the block into shared memory (cp.async), then into tensor memory; read panel 0
//   into registers (each thread: its complex row r = 32 w + lane, and in warps 0-1 half of
//   one tile-2 row);
//   for each panel P: factor it (one CTA barrier per pivot) while the rest of update P - 1
//   runs; once update P - 1 is complete, write panel P back, zero its pivot rows elsewhere
//   while collecting R, stage A and B in shared memory, issue update P's MMAs for the
//   columns of panel P + 1 (commit) and then for the rest (commit); wait for the first
//   commit and read panel P + 1;
//   after the last update, write the inverse out through shared memory with both
//   permutations applied.
// Every wait is bounded (limit passed in); on expiry the kernel records DEV_TIMEOUT, waits
// (bounded, at the default limit) for its own MMAs, frees tensor memory and returns.
#include "common.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int GJT_PWARPS = 6;                        // panel warps
constexpr int GJT_PTHREADS = 32 * GJT_PWARPS;
constexpr int GJT_THREADS = GJT_PTHREADS + 32;       // + one MMA-issue warp
constexpr int GJT_NB = 16;                           // panel width (complex columns)
constexpr int GJT_NMAX = 160;
constexpr int GJT_K = 2 * GJT_NB;                    // real K of a panel update
constexpr uint32_t GJT_LBO = 128;                    // next core matrix along K
constexpr uint32_t GJT_SBO = (GJT_K / 4) * 128;      // next 8-row group: 1024 bytes
constexpr uint32_t GJT_ATILE = 128 * GJT_K * 4;      // one split of one A tile: 16 KB
constexpr uint32_t GJT_BSPLIT = GJT_NMAX * GJT_K * 4;  // one split of B: 20 KB
constexpr int GJT_RLD = GJT_NMAX + 4;                // R staging row stride (floats)
constexpr int GJT_SLD = 2 * GJT_NMAX + 4;            // block staging row stride (floats):
                                                     // 16 bytes past a multiple of 128
// shared memory: block staging (load and store), overlaid while factoring by A, B and R
constexpr size_t GJT_STAGE = (size_t)GJT_NMAX * GJT_SLD * 4;          // 207,360
constexpr size_t GJT_A_OFF = 0;                                        // 3 tiles x hi, lo
constexpr size_t GJT_B_OFF = GJT_A_OFF + 6 * (size_t)GJT_ATILE;        // hi, lo
constexpr size_t GJT_R_OFF = GJT_B_OFF + 2 * (size_t)GJT_BSPLIT;
constexpr size_t GJT_R_END = GJT_R_OFF + (size_t)GJT_K * GJT_RLD * 4;
static_assert(GJT_R_END <= GJT_STAGE, "operands overlay the staging area");
static_assert(GJT_B_OFF % 1024 == 0 && GJT_R_OFF % 16 == 0, "operand alignment");
// small region after the staging area
constexpr size_t GJT_PIV_OFF = GJT_STAGE;                              // int[160]
constexpr size_t GJT_PINV_OFF = GJT_PIV_OFF + GJT_NMAX * 4;            // int[160]
constexpr size_t GJT_ROW_OFF = GJT_PINV_OFF + GJT_NMAX * 4;            // float2[2][6][16]
constexpr size_t GJT_SLOTK_OFF = GJT_ROW_OFF + 2 * GJT_PWARPS * 16 * 8;  // uint64[2]
constexpr size_t GJT_BAR_OFF = GJT_SLOTK_OFF + 2 * 8;                  // 4 mbarriers
constexpr size_t GJT_SLOT_OFF = GJT_BAR_OFF + 4 * 8;                   // tmem address, abort
constexpr size_t GJT_SMEM = GJT_SLOT_OFF + 16;
static_assert(GJT_SMEM <= 227 * 1024, "fits one CTA per SM");
static_assert(GJT_ROW_OFF % 16 == 0 && GJT_SLOTK_OFF % 8 == 0, "alignment of the small region");

constexpr long long GJT_DEFAULT_WAIT = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of real element (row, k) of a K-major, no-swizzle operand with K = 32
__device__ __forceinline__ uint32_t kmaj_off(int row, int k) {
  return (uint32_t)(row >> 3) * GJT_SBO + (uint32_t)(k >> 2) * GJT_LBO + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 3) * 4u;
}

__device__ __forceinline__ uint64_t kmaj_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((GJT_LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((GJT_SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle
  return d;
}

// TF32 hi part rounded to nearest (ties away), lo = x - hi exact (as in the GEMM)
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  lo = x - hi;
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, 1, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// barrier 1 among the panel warps only (the MMA warp does not take part)
__device__ __forceinline__ void pbar() {
  asm volatile("bar.sync 1, %0;" ::"r"(GJT_PTHREADS) : "memory");
}
__device__ __forceinline__ bool pbar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(GJT_PTHREADS)
      : "memory");
  return r != 0u;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar))
      : "memory");
}

// bounded wait taken by a whole warp together (no lane parked at a shuffle while one lane
// polls, which costs several hundred cycles per wait), ending early when another warp has
// given up: the phase has completed once any
// lane sees it complete; the warp gives up together on the abort flag or the limit
__device__ __forceinline__ bool warp_wait_ab(uint64_t* bar, uint32_t parity, long long limit,
                                             volatile int* abort_flag) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (__any_sync(0xffffffffu, done != 0u)) return true;
    const bool expired = clock64() - t0 > limit;
    if (__any_sync(0xffffffffu, expired || *abort_flag != 0)) {
      if (expired) *abort_flag = 1;
      return false;
    }
  }
}

// 1 / (re + i im) = (re - i im) / (re^2 + im^2).  Both parts are scaled by the power of two
// that brings the larger magnitude into [1, 2) (exact), so d = ar^2 + ai^2 lies in [1, 8);
// 1 / d is the hardware approximation refined by one Newton step r <- r + r (1 - d r), and
// the result is scaled back.  Returns 0 when the larger magnitude is below 1e-37 (a zero
// pivot in FP32 terms) or not finite.
__device__ __forceinline__ float2 crecip_fast(float re, float im) {
  const float s = fmaxf(fabsf(re), fabsf(im));
  if (!(s > 1e-37f) || !(s < 1e37f)) return make_float2(0.f, 0.f);
  const uint32_t e = __float_as_uint(s) & 0x7F800000u;
  const float sc = __uint_as_float(0x7F000000u - e);   // 2^-(exponent of s), exact
  const float ar = re * sc, ai = im * sc;
  const float d = fmaf(ar, ar, ai * ai);
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  r = fmaf(r, fmaf(-d, r, 1.f), r);
  const float q = r * sc;
  return make_float2(ar * q, -ai * q);
}

constexpr uint32_t idesc_n(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

struct GjtArgs {
  const float2* src;
  int64_t src_stride;   // complex elements between blocks
  float2* out;
  int64_t out_stride;
  int n, batch;
  int32_t* status;
  long long wait_limit;
  int vec16;            // 1: rows may be copied in 16-byte pieces (n even, 16-byte aligned)
  uint32_t* maxabs;     // or null: atomicMax of the bits of the largest |re|, |im| read
};

// Threads and rows: panel warps 0-3 own complex rows r = 32 w + lane (tiles 0 and 1, their
// lane quarter); panel warps 4-5 own rows r = 128 + 16 (w - 4) + lane for lanes < 16 (tile 2,
// lane quarter w - 4: real part in that lane, imaginary part 16 lanes up).  Each thread
// keeps the 16 panel columns of its row in registers, both parts.  Warp 6 issues the MMAs:
// the panel warps arrive on "ops" when the operands of an update are staged, warp 6 issues
// the update and commits it to "head" (the next panel's columns) and "bulk" (the rest).
__global__ void __launch_bounds__(GJT_THREADS, 1) tc_gj_kernel(GjtArgs p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  float* stage = reinterpret_cast<float*>(sm);
  unsigned char* Ahi = sm + GJT_A_OFF;                         // tile tau: + tau * ATILE
  unsigned char* Alo = sm + GJT_A_OFF + 3 * GJT_ATILE;
  unsigned char* Bhi = sm + GJT_B_OFF;
  unsigned char* Blo = sm + GJT_B_OFF + GJT_BSPLIT;
  float* Rst = reinterpret_cast<float*>(sm + GJT_R_OFF);
  int* piv = reinterpret_cast<int*>(sm + GJT_PIV_OFF);
  int* pinv = reinterpret_cast<int*>(sm + GJT_PINV_OFF);
  float2* rowbuf = reinterpret_cast<float2*>(sm + GJT_ROW_OFF);  // [2][GJT_PWARPS][16]
  unsigned long long* pslot = reinterpret_cast<unsigned long long*>(sm + GJT_SLOTK_OFF);  // [2]
  uint64_t* bar_head = reinterpret_cast<uint64_t*>(sm + GJT_BAR_OFF);
  uint64_t* bar_bulk = bar_head + 1;
  uint64_t* bar_ops = bar_head + 2;
  uint64_t* bar_done = bar_head + 3;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + GJT_SLOT_OFF);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + GJT_SLOT_OFF + 4);

  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int n = p.n;
  const int np = (n + GJT_NB - 1) / GJT_NB * GJT_NB;
  const int T = np > 128 ? 3 : 2;                 // tensor-memory tiles
  const int TS = T == 3 ? 160 : 128;              // columns per tile
  const uint32_t tcols = T == 3 ? 512u : 256u;
  const int npanel = np / GJT_NB;
  const int SLD = 2 * np + 4;                     // staging row stride for this size (floats)
  constexpr uint32_t FULL = 0xffffffffu;

  // this thread's row and where its parts live
  const bool mma_warp = w == GJT_PWARPS;
  const bool main_warp = w < 4;                   // tiles 0 / 1
  const int row = main_warp ? 32 * w + l : 128 + 16 * (w - 4) + (l & 15);
  const bool hasrow = main_warp ? row < np : (!mma_warp && T == 3 && l < 16 && row < np);
  const int part = main_warp ? 0 : (l >> 4);      // tile 2: 0 real lane, 1 imaginary lane
  const bool tile2_lane = !main_warp && !mma_warp && T == 3 && row < np;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar_head)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar_bulk)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar_ops)),
                 "r"(GJT_PWARPS));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar_done)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)(32 * (w & 3)) << 16;
  auto taddr = [&](int tile, int col) -> uint32_t {
    return tmem + lane_base + (uint32_t)(tile * TS + col);
  };

  uint32_t nhead = 0, nbulk = 0, nops = 0;   // completed phases of the barriers
  bool ok = true, sing = false, mma_issued = false;

  for (int blk = blockIdx.x; blk < p.batch && ok; blk += gridDim.x) {
    // ------------------------------------------------ block -> staging (identity padding)
    const float2* g = p.src + (int64_t)blk * p.src_stride;
    if (p.vec16) {
      const int halfn = n >> 1;
      for (int e = tid; e < n * halfn; e += GJT_THREADS) {
        const int r = e / halfn, c2 = e - r * halfn;
        const uint32_t dst = smem_u32(stage + r * SLD + 4 * c2);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                     "l"(g + (int64_t)r * n + 2 * c2)
                     : "memory");
      }
    } else {
      for (int e = tid; e < n * n; e += GJT_THREADS) {
        const int r = e / n, c = e - r * n;
        const uint32_t dst = smem_u32(stage + r * SLD + 2 * c);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst),
                     "l"(g + (int64_t)r * n + c)
                     : "memory");
      }
    }
    if (np != n) {
      for (int e = tid; e < np * np; e += GJT_THREADS) {
        const int r = e / np, c = e - r * np;
        if (r >= n || c >= n)
          *reinterpret_cast<float2*>(stage + r * SLD + 2 * c) =
              make_float2(r == c ? 1.f : 0.f, 0.f);
      }
    }
    if (tid == 0) pslot[0] = pslot[1] = 0ull;
    // the next block of this CTA into L2 while this one is factored
    if (blk + (int)gridDim.x < p.batch) {
      const char* nb = reinterpret_cast<const char*>(p.src + (int64_t)(blk + gridDim.x) * p.src_stride);
      for (int e = tid; e < (n * n * 8 + 127) / 128; e += GJT_THREADS)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(nb + (int64_t)e * 128));
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // ------------------------------------------------ staging -> tensor memory
    if (main_warp) {
      float amax = 0.f;
      for (int c0 = 0; c0 < np; c0 += 16) {
        float re[16], im[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4 v = hasrow ? *reinterpret_cast<const float4*>(stage + row * SLD + 2 * c0 + 4 * q)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
          re[2 * q] = v.x;
          im[2 * q] = v.y;
          re[2 * q + 1] = v.z;
          im[2 * q + 1] = v.w;
          amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        tmem_st16(taddr(0, c0), re);
        tmem_st16(taddr(1, c0), im);
      }
      // the largest magnitude of the block (rows 128 .. 159 are read by warps 4-5 as well,
      // but those are covered here too: warps 0-3 see every row < 128, the tile-2 warps below)
      if (p.maxabs) {
        const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(amax));
        if (l == 0) atomicMax(p.maxabs, m);
      }
    } else if (!mma_warp && T == 3) {
      for (int c0 = 0; c0 < np; c0 += 16) {
        float y[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4 v = tile2_lane ? *reinterpret_cast<const float4*>(stage + row * SLD + 2 * c0 + 4 * q)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
          y[2 * q] = part ? v.y : v.x;
          y[2 * q + 1] = part ? v.w : v.z;
        }
        tmem_st16(taddr(2, c0), y);
      }
      if (p.maxabs) {
        float amax = 0.f;
        for (int c0 = 0; tile2_lane && part == 0 && c0 < np; c0 += 2) {
          const float4 v = *reinterpret_cast<const float4*>(stage + row * SLD + 2 * c0);
          amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(amax));
        if (l == 0) atomicMax(p.maxabs, m);
      }
    }
    tmem_wait_st();
    fence_before();
    __syncthreads();
    fence_after();

    if (mma_warp) {
      // ---------------------------------------------- MMA issue (the warp waits, one lane issues)
      {
        const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo);
        const uint32_t bh = smem_u32(Bhi), bl = smem_u32(Blo);
        auto range = [&](int j0, int j1) {
          const uint32_t idesc = idesc_n(j1 - j0);
          for (int tile = 0; tile < T; ++tile) {
            const uint32_t d = tmem + (uint32_t)(tile * TS + j0);
#pragma unroll
            for (int ks = 0; ks < GJT_K / 8; ++ks) {
              const uint32_t ao = (uint32_t)tile * GJT_ATILE + (uint32_t)ks * 2 * GJT_LBO;
              const uint32_t bo = (uint32_t)(j0 >> 3) * GJT_SBO + (uint32_t)ks * 2 * GJT_LBO;
              mma_tf32(d, kmaj_desc(ah + ao), kmaj_desc(bh + bo), idesc);
              mma_tf32(d, kmaj_desc(ah + ao), kmaj_desc(bl + bo), idesc);
              mma_tf32(d, kmaj_desc(al + ao), kmaj_desc(bh + bo), idesc);
            }
          }
        };
        for (int P = 0; P < npanel; ++P) {
          const int c0 = P * GJT_NB;
          const bool has_next = P + 1 < npanel;
          const int h1 = has_next ? c0 + 2 * GJT_NB : c0 + GJT_NB;
          const bool bulk_lo = c0 > 0, bulk_hi = h1 < np;
          if (!warp_wait_ab(bar_ops, nops & 1u, p.wait_limit, abort_flag)) {
            ok = false;
            break;
          }
          ++nops;
          fence_after();
          if (l == 0) {
            if (has_next) {
              range(c0 + GJT_NB, h1);
              mma_commit(bar_head);
            }
            if (bulk_lo) range(0, c0);
            if (bulk_hi) range(h1, np);
            if (bulk_lo || bulk_hi) mma_commit(bar_bulk);
            if (has_next || bulk_lo || bulk_hi) mma_issued = true;
          }
          __syncwarp();
        }
      }
      __syncwarp();
    } else {
      // ---------------------------------------------- panel warps
      float xr[16], xi[16];
      bool used = !hasrow;
      auto read_panel = [&](int c0) {
        if (main_warp) {
          tmem_ld16(taddr(0, c0), xr);
          tmem_ld16(taddr(1, c0), xi);
          tmem_wait_ld();
        } else if (T == 3) {
          float v[16];
          tmem_ld16(taddr(2, c0), v);
          tmem_wait_ld();
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            xr[t] = v[t];
            xi[t] = __shfl_sync(FULL, v[t], (l & 15) + 16);
          }
        }
        if (!hasrow) {
#pragma unroll
          for (int t = 0; t < 16; ++t) xr[t] = xi[t] = 0.f;
        }
      };
      // this thread's tensor-memory values of the panel columns (both parts, or this lane's)
      auto write_panel = [&](int c0) {
        if (main_warp) {
          tmem_st16(taddr(0, c0), xr);
          tmem_st16(taddr(1, c0), xi);
        } else if (T == 3) {
          float v[16];
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const float im = __shfl_sync(FULL, xi[t], l & 15);
            v[t] = part ? im : xr[t];
          }
          tmem_st16(taddr(2, c0), v);
        }
      };
      // each warp waits (bounded, abort-aware) as a whole, then the panel warps agree
      auto wait_all = [&](uint64_t* bar, uint32_t& cnt) -> bool {
        const bool got = warp_wait_ab(bar, cnt & 1u, p.wait_limit, abort_flag);
        ++cnt;
        const bool all = pbar_and(got);
        fence_after();
        return all;
      };

      // Gauss-Jordan steps on the panel, one barrier (of the panel warps) each, four steps
      // per loop iteration with the pivot column at x[u]; after each group the registers
      // rotate by four, so after the panel the columns are back in order.
      // Pivot election: a 32-bit key per candidate row, the bits of |re| + |im| with the low
      // 8 mantissa bits replaced by 255 - row (the largest magnitude to 2^-15 relative, ties
      // to the lowest row), reduced over the warp, then one 64-bit shared-memory atomicMax per
      // warp of (step + 1) << 32 | key: older steps always lose, so the two slots (by step
      // parity) need clearing only per block.  The warp's winning lane publishes its row.
      // The election of step k + 1 runs inside step k, right after the next pivot column is
      // updated, so its latency hides under the update of the other columns.
      auto pkey = [&](float re, float im) -> uint32_t {
        const float m = fabsf(re) + fabsf(im);
        const uint32_t bits = m >= 0.f ? (__float_as_uint(m) & 0xFFFFFF00u) : 0u;
        return bits | (255u - (uint32_t)row);
      };
      auto publish = [&](int b) {
        float4* rb = reinterpret_cast<float4*>(rowbuf + (b * GJT_PWARPS + w) * 16);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          rb[q] = make_float4(xr[2 * q], xi[2 * q], xr[2 * q + 1], xi[2 * q + 1]);
      };
      auto factor_panel = [&](int c0) {
        {  // election of the panel's first pivot
          const uint32_t key = used ? 0u : pkey(xr[0], xi[0]);
          const uint32_t kmax = __reduce_max_sync(FULL, key);
          if (l == 0)
            atomicMax(&pslot[c0 & 1], ((unsigned long long)(c0 + 1) << 32) | kmax);
          if (!used && key == kmax) publish(c0 & 1);
        }
#pragma unroll 1
        for (int g4 = 0; g4 < GJT_NB; g4 += 4) {
          bool win_next = false;  // this lane publishes the pivot row of the next group's step
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int k = c0 + g4 + u, b = k & 1;
            const bool last = g4 + u == GJT_NB - 1;
            pbar();
            const unsigned long long v = pslot[b];
            const int P = 255 - (int)(v & 255ull);
            const int W = P < 128 ? (P >> 5) : 4 + ((P - 128) >> 4);
            if (tid == 0) piv[k] = P;
            float rr[16], ri[16];
            const float4* rb = reinterpret_cast<const float4*>(rowbuf + (b * GJT_PWARPS + W) * 16);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float4 x4 = rb[q];
              rr[2 * q] = x4.x;
              ri[2 * q] = x4.y;
              rr[2 * q + 1] = x4.z;
              ri[2 * q + 1] = x4.w;
            }
            const float2 pinv = crecip_fast(rr[u], ri[u]);
            if (tid == 0 && (((uint32_t)v >> 8) == 0u || (pinv.x == 0.f && pinv.y == 0.f)))
              sing = true;
            // pivot row: row / pivot with 1 / pivot in the pivot column; other rows:
            // x - (x_u / pivot) row with -x_u / pivot in the pivot column
            const bool isp = !used && row == P;
            const float2 f = make_float2(xr[u], xi[u]) * pinv;
            const float2 a = isp ? pinv : make_float2(-f.x, -f.y);
            if (isp) used = true;
            auto upd = [&](int t) {
              const float2 base = isp ? make_float2(0.f, 0.f) : make_float2(xr[t], xi[t]);
              const float2 nv = cfma(a, make_float2(rr[t], ri[t]), base);
              xr[t] = nv.x;
              xi[t] = nv.y;
            };
            // the next pivot column first, and the next election
            const int nx = u + 1;
            upd(nx);
            uint32_t key2 = 0, kmax2 = 0;
            if (!last) {
              key2 = used ? 0u : pkey(xr[nx], xi[nx]);
              kmax2 = __reduce_max_sync(FULL, key2);
              if (l == 0)
                atomicMax(&pslot[b ^ 1], ((unsigned long long)(k + 2) << 32) | kmax2);
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              if (t == nx) continue;
              if (t == u) {
                xr[t] = a.x;
                xi[t] = a.y;
              } else {
                upd(t);
              }
            }
            // the row is published in the order the readers will hold: after the rotation
            // below when the next step opens the next group
            if (u < 3) {
              if (!last && !used && key2 == kmax2) publish(b ^ 1);
            } else {
              win_next = !last && !used && key2 == kmax2;
            }
          }
          float tr[4], ti[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            tr[t] = xr[t];
            ti[t] = xi[t];
          }
#pragma unroll
          for (int t = 0; t < 12; ++t) {
            xr[t] = xr[t + 4];
            xi[t] = xi[t + 4];
          }
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            xr[12 + t] = tr[t];
            xi[12 + t] = ti[t];
          }
          if (win_next) publish((c0 + g4 + 4) & 1);
        }
      };

      // Iteration P: factor panel P (its columns already hold update P - 1) while the rest
      // of update P - 1 runs; then, with update P - 1 complete, write panel P back, collect
      // R, stage the operands and hand them to the MMA warp; read panel P + 1 once its
      // columns are updated.
      bool pending_bulk = false;
      read_panel(0);
      for (int P = 0; P < npanel; ++P) {
        const int c0 = P * GJT_NB;
        const bool has_next = P + 1 < npanel;
        const int h1 = has_next ? c0 + 2 * GJT_NB : c0 + GJT_NB;
        const bool bulk_lo = c0 > 0, bulk_hi = h1 < np;
        factor_panel(c0);
        if (pending_bulk) {
          pending_bulk = false;
          if (!wait_all(bar_bulk, nbulk)) {
            ok = false;
            break;
          }
        } else {
          pbar();  // piv[] of this panel is visible
        }
        // ---- write panel P, zero its pivot rows elsewhere and collect R
        int u0 = -1;
        if (hasrow) {
#pragma unroll 4
          for (int u = 0; u < GJT_NB; ++u)
            if (piv[c0 + u] == row) u0 = u;
        }
        write_panel(c0);
        // R rows: k = 2 u + (0 real, 1 imaginary) for pivot u of this panel
        int ku0 = -1, ku1 = -1;  // main warps: tiles 0 and 1; tile-2 warps: their lane's part
        if (main_warp) {
          if (u0 >= 0) {
            ku0 = 2 * u0;
            ku1 = 2 * u0 + 1;
          }
        } else {
          const int up = __shfl_sync(FULL, u0, l & 15);
          ku0 = (T == 3 && up >= 0) ? 2 * up + part : -1;
        }
        const int ntile = main_warp ? 2 : (T == 3 ? 1 : 0);
        for (int i = 0; i < ntile; ++i) {
          const int tile = main_warp ? i : 2;
          const int ku = i == 0 ? ku0 : ku1;
          if (__ballot_sync(FULL, ku >= 0) == 0u) continue;
          for (int j0 = 0; j0 < np; j0 += 32) {
            // two 16-column chunks per round trip (panel P's chunk is skipped)
            const bool a_ok = j0 != c0, b_ok = j0 + 16 < np && j0 + 16 != c0;
            float va[16], vb[16];
            if (a_ok) tmem_ld16(taddr(tile, j0), va);
            if (b_ok) tmem_ld16(taddr(tile, j0 + 16), vb);
            tmem_wait_ld();
            if (ku >= 0) {
              if (a_ok) {
                float4* dst = reinterpret_cast<float4*>(Rst + ku * GJT_RLD + j0);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  dst[q] = make_float4(va[4 * q], va[4 * q + 1], va[4 * q + 2], va[4 * q + 3]);
              }
              if (b_ok) {
                float4* dst = reinterpret_cast<float4*>(Rst + ku * GJT_RLD + j0 + 16);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  dst[q] = make_float4(vb[4 * q], vb[4 * q + 1], vb[4 * q + 2], vb[4 * q + 3]);
              }
#pragma unroll
              for (int t = 0; t < 16; ++t) va[t] = vb[t] = 0.f;
            }
            if (a_ok) tmem_st16(taddr(tile, j0), va);
            if (b_ok) tmem_st16(taddr(tile, j0 + 16), vb);
          }
        }
        tmem_wait_st();
        // ---- A: the factored panel in stacked form, TF32 hi / lo.  Row (r, Re) = (Re, -Im)
        // pairs, row (r, Im) = (Im, Re) pairs over the 16 panel columns.
        if (hasrow) {
          const int tre = main_warp ? 0 : 2, tim = main_warp ? 1 : 2;
          const int lre = main_warp ? row : 32 * (w - 4) + l;      // lanes within the tiles
          const int lim = main_warp ? row : 32 * (w - 4) + l + 16;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int ua = 2 * q, ub = 2 * q + 1;
            const float vr[4] = {xr[ua], -xi[ua], xr[ub], -xi[ub]};
            const float vi[4] = {xi[ua], xr[ua], xi[ub], xr[ub]};
            float h[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) split_tf32(vr[e], h[e], lo[e]);
            const uint32_t ore = (uint32_t)tre * GJT_ATILE + kmaj_off(lre, 4 * q);
            *reinterpret_cast<float4*>(Ahi + ore) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4*>(Alo + ore) = make_float4(lo[0], lo[1], lo[2], lo[3]);
#pragma unroll
            for (int e = 0; e < 4; ++e) split_tf32(vi[e], h[e], lo[e]);
            const uint32_t oim = (uint32_t)tim * GJT_ATILE + kmaj_off(lim, 4 * q);
            *reinterpret_cast<float4*>(Ahi + oim) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4*>(Alo + oim) = make_float4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
        pbar();  // R complete
        // ---- B: R in K-major form, TF32 hi / lo (columns of panel P are not used); lanes
        // take consecutive columns, so the reads of R and the stores of B are conflict-free
        for (int e = tid; e < np * 8; e += GJT_PTHREADS) {
          const int q = e / np, col = e - q * np;
          if (col >= c0 && col < c0 + GJT_NB) continue;
          float h[4], lo[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) split_tf32(Rst[(4 * q + i) * GJT_RLD + col], h[i], lo[i]);
          const uint32_t o = kmaj_off(col, 4 * q);
          *reinterpret_cast<float4*>(Bhi + o) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(Blo + o) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
        // operands (generic-proxy stores) and the tensor-memory stores above, handed to the
        // MMA warp
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncwarp();
        if (l == 0) mbar_arrive(bar_ops);
        pending_bulk = bulk_lo || bulk_hi;
        if (has_next) {
          if (!wait_all(bar_head, nhead)) {
            ok = false;
            break;
          }
          read_panel(c0 + GJT_NB);
        }
      }
      if (ok && pending_bulk) {
        if (!wait_all(bar_bulk, nbulk)) ok = false;
      }
    }
    ok = __syncthreads_and(ok) && !*abort_flag;
    if (!ok) break;
    fence_after();
    // ------------------------------------------------ inverse out: M[piv[i]][pinv[j]]
    // through the staging area (free again), then coalesced row stores
    for (int e = tid; e < np; e += GJT_THREADS) pinv[piv[e]] = e;
    __syncthreads();
    if (!mma_warp) {
      const int io = hasrow ? pinv[row] : n;
      for (int j0 = 0; j0 < np; j0 += 16) {
        float re[16], im[16];
        if (main_warp) {
          tmem_ld16(taddr(0, j0), re);
          tmem_ld16(taddr(1, j0), im);
          tmem_wait_ld();
        } else if (T == 3) {
          tmem_ld16(taddr(2, j0), re);
          tmem_wait_ld();
#pragma unroll
          for (int t = 0; t < 16; ++t) im[t] = __shfl_sync(FULL, re[t], (l & 15) + 16);
        }
        if (hasrow && io < n) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int jo = piv[j0 + t];
            if (jo < n)
              *reinterpret_cast<float2*>(stage + io * SLD + 2 * jo) = make_float2(re[t], im[t]);
          }
        }
      }
    }
    fence_before();
    __syncthreads();
    fence_after();
    float2* o = p.out + (int64_t)blk * p.out_stride;
    for (int e = tid; e < n * n; e += GJT_THREADS) {
      const int i = e / n, j = e - i * n;
      o[e] = *reinterpret_cast<const float2*>(stage + i * SLD + 2 * j);
    }
    __syncthreads();
  }
  if (!ok && tid == 0) atomicCAS(p.status, DEV_OK, DEV_TIMEOUT);
  if (sing && tid == 0) atomicCAS(p.status, DEV_OK, DEV_SINGULAR);
  // every MMA this CTA issued has finished before its tensor memory is freed
  if (mma_warp && l == 0 && mma_issued) {
    mma_commit(bar_done);
    if (!mbar_wait(bar_done, 0, GJT_DEFAULT_WAIT)) atomicCAS(p.status, DEV_OK, DEV_TIMEOUT);
  }
  fence_before();
  __syncthreads();
  if (w == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols)
                 : "memory");
  }
}

}  // namespace

cudaError_t launch_tc_gj(const float2* src, int64_t src_stride, float2* out, int64_t out_stride,
                         int n, int batch, int32_t* status, cudaStream_t s, uint32_t* maxabs) {
  if (batch <= 0) return cudaSuccess;
  if (n < 1 || n > GJT_NMAX) return cudaErrorInvalidValue;
  static const cudaError_t attr = cudaFuncSetAttribute(
      tc_gj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GJT_SMEM);
  RCI_CUDA_TRY(attr);
  int dev = 0, nsm = 0;
  RCI_CUDA_TRY(cudaGetDevice(&dev));
  RCI_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  GjtArgs a{src, src_stride, out, out_stride, n, batch, status, tc_wait_limit(), 0, maxabs};
  a.vec16 = (n % 2 == 0) && ((uintptr_t)src % 16 == 0) && (src_stride % 2 == 0);
  const int grid = batch < nsm ? batch : nsm;
  tc_gj_kernel<<<grid, GJT_THREADS, GJT_SMEM, s>>>(a);
  rci_note_launch();
  return cudaGetLastError();
}
