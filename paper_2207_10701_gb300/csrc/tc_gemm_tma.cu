// Batched complex FP32 GEMM on the 5th-generation tensor cores, fed by the Tensor Memory
// Accelerator, with the A operand in tensor memory (3xTF32, real alpha and beta):
//
//   C[z] = alpha op(A[z]) op(B[z]) + beta C0[z]      (row-major complex64, N <= 160)
//
// Algebra (as the shared-memory kernels in tc_gemm.cu): the complex product is the real
// product of the stacked A_s (rows (ar, -ai) and (ai, ar) per complex k) with B_s (rows
// br, bi per complex k), each FP32 operand split into TF32 hi + lo and three MMAs per K step
// (hi hi, hi lo, lo hi) accumulating in FP32.  Here the two stacked rows of complex row l
// are interleaved: tensor-memory lane 2 l holds Re C[l][:], lane 2 l + 1 holds Im C[l][:],
// so a 128-lane tile covers 64 complex rows and the epilogue pairs Re and Im with one
// shuffle between neighbouring lanes.
//
// Why this layout.  With both operands in shared memory a 128 x 160 x 8 MMA reads 9 KB of
// shared memory, and the split operands have to be written there first: about 90 KB per
// K stage against the 128 bytes per clock an SM's shared memory delivers, which caps the
// shared-memory kernel near 70 % of the TF32 rate before any latency.  With A in tensor
// memory the MMAs read only B (5 KB each), and the raw tiles arrive by TMA, so no warp
// holds global loads in flight.
//
// Roles of one persistent CTA (one per SM, 14 warps), over the CTA's tiles (tile = product
// z x 64-row block) and their K stages of 8 complex k:
//   warp 12    TMA: raw A (64 rows x 8 k, or 8 k x 64 rows for op = T) and raw B (8 k x N,
//              or N x 8 k) into a ring of raw stages, completion by mbarrier transaction
//              count (one lane issues);
//   warps 0-7  convert, in two groups of four that take the stages in turn: warp w writes
//              tensor-memory lanes 32 (w % 4) .. + 31: each lane builds its stacked row,
//              splits it and stores hi and lo into the stage's tensor-memory A slot
//              (tcgen05.st); the group's threads split B (five items each) into the stage's
//              shared-memory slot (K-major core matrices), all loads before the stores;
//   warp 13    waits for a converted stage; one lane issues its six MMAs (A from tensor
//              memory, B from shared memory) and commits them to the stage's "empty"
//              barrier; after a tile, to the accumulator's "full" barrier;
//   warps 8-11 epilogue: read 16 accumulator columns at a time (warp w: lanes
//              32 (w % 4) ..), exchange Re / Im with the neighbouring lane and store
//              16-byte pieces (two complex) so that each lane pair writes one full 32-byte
//              sector; C0 of the next chunk is loaded while the current one is stored.
// Every role waits as a whole warp (a lane-0 poll with the other lanes parked at a shuffle
// costed several hundred cycles per wait, even on a completed barrier).
// Two accumulators (tensor-memory columns 0 and 256) let a tile's epilogue run under the
// next tile's MMAs; the converted-stage A slots sit in the columns between.
// Every wait is bounded; the first that runs out sets a shared abort flag that ends the
// others; the kernel records DEV_TIMEOUT, waits (bounded) for its own TMA copies and MMAs,
// frees its tensor memory and returns.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int TT_ROWS = 64;       // complex rows per tile (128 tensor-memory lanes)
constexpr int TT_KC = 8;          // complex k per stage
constexpr int TT_NMAX = 160;      // largest N (complex columns)
#ifndef RCI_TMA_RAW_STAGES
#define RCI_TMA_RAW_STAGES 4
#endif
#ifndef RCI_TMA_CONV_STAGES
#define RCI_TMA_CONV_STAGES 4
#endif
constexpr int TT_RS = RCI_TMA_RAW_STAGES;    // raw stages (TMA in flight)
constexpr int TT_CS = RCI_TMA_CONV_STAGES;   // converted stages (tensor-memory A slot + B)
// Eight converter warps in TT_GROUPS groups that take the K stages in turn (group g the
// stages it with it % TT_GROUPS == g), so that one group's waits and fences overlap the
// other's work; a group has a warp (or two) per tensor-memory lane quarter.
#ifndef RCI_TMA_CONV_GROUPS
#define RCI_TMA_CONV_GROUPS 2
#endif
constexpr int TT_GROUPS = RCI_TMA_CONV_GROUPS;
constexpr int TT_CONV_WARPS = 8, TT_EPI_WARP0 = 8, TT_TMA_WARP = 12, TT_MMA_WARP = 13;
constexpr int TT_THREADS = 14 * 32;
constexpr int TT_GWARPS = TT_CONV_WARPS / TT_GROUPS;      // warps per group
constexpr int TT_GTHREADS = 32 * TT_GWARPS;
constexpr int TT_KSPLIT = TT_GWARPS / 4;                  // warps per lane quarter in a group
constexpr int TT_BITEMS = (TT_NMAX * 4 + TT_GTHREADS - 1) / TT_GTHREADS;
static_assert(TT_GWARPS % 4 == 0 && (TT_KSPLIT == 1 || TT_KSPLIT == 2), "group shape");
constexpr uint32_t TT_RAW_A = TT_ROWS * TT_KC * 8;        // 4096 bytes
constexpr uint32_t TT_RAW_B = TT_NMAX * TT_KC * 8;        // 10240 bytes (N = 160)
constexpr uint32_t TT_RAW_STAGE = TT_RAW_A + TT_RAW_B;    // 14336 = 14 x 1024
constexpr uint32_t TT_LBO = 128;                          // next core matrix along K
constexpr uint32_t TT_SBO = (2 * TT_KC / 4) * 128;        // next 8-row group: 512 bytes
constexpr uint32_t TT_BSPLIT = TT_NMAX * 2 * TT_KC * 4;   // one split of B: 10240 bytes
constexpr uint32_t TT_CSTAGE = 2 * TT_BSPLIT;
constexpr size_t TT_CONV_OFF = (size_t)TT_RS * TT_RAW_STAGE;
constexpr size_t TT_BAR_OFF = TT_CONV_OFF + (size_t)TT_CS * TT_CSTAGE;
constexpr int TT_NBAR = 2 * TT_RS + 2 * TT_CS + 2 + 2 + 1;
constexpr size_t TT_SMEM = TT_BAR_OFF + (size_t)TT_NBAR * 8 + 16;
static_assert(TT_RAW_STAGE % 1024 == 0 && TT_RAW_A % 1024 == 0, "swizzled TMA destinations");
static_assert(TT_CONV_OFF % 1024 == 0 && TT_CSTAGE % 1024 == 0, "operand alignment");
static_assert(TT_SMEM <= 227 * 1024, "one CTA per SM");
static_assert(TT_NMAX * 4 <= TT_BITEMS * TT_GTHREADS, "B items per converter thread");
// tensor-memory columns: accumulators, then the A slots (hi in 16 columns, lo in the next 16)
constexpr uint32_t TT_TMEM_COLS = 512;
constexpr uint32_t TT_ACC_STRIDE = 256;  // accumulator b at column 256 b
__device__ __forceinline__ uint32_t a_slot(int cs) {
  return cs < 3 ? 160u + 32u * (uint32_t)cs : 416u + 32u * (uint32_t)(cs - 3);
}
static_assert(TT_CS <= 6, "six A slots fit beside the accumulators");
constexpr long long TT_DEFAULT_WAIT = 4000000000LL;

// A launch runs up to two jobs (independent sets of products with their own operands and
// outputs, e.g. X = Dinv L and Y = Dinv L^T of one reduction level), their tiles numbered job
// after job.  A product may run over up to two K segments with their own operands (the Schur
// update D - L_2k Y_k-1 - L_2k+1^T X_k as one product over K = 2 ny): segment g of output z
// reads A member z + zA and B member z + zB of its tensor maps, for zlo <= z < zhi only.
struct TtSeg {
  int nkb;          // K stages (8 complex k each)
  int zA, zB;       // batch offsets of its operands
  int zlo, zhi;     // outputs that include this segment
  int ta, tb;       // op(A), op(B): 1 = transpose
};

struct TtJob {
  int batch, nseg, tile0;  // tile0: the job's first tile in the launch
  TtSeg seg[2];
  float2* C;
  int64_t ldc, sC;
  const float2* C0;
  int64_t ldc0, sC0;
  float alpha, beta;
};

struct TtArgs {
  int M, N, NB;     // NB: N rounded up to 16 (the MMA's N)
  int njob, ntiles;
  TtJob job[2];
  int32_t* status;
  long long wait_limit;
};

// tensor maps: job j, segment g: A at 4 j + 2 g, B at 4 j + 2 g + 1
struct TtMaps {
  CUtensorMap m[8];
};

// the address of map i, each one a constant offset into the parameter
__device__ __forceinline__ const CUtensorMap* map_at(const TtMaps& maps, int i) {
  switch (i) {
    case 0: return &maps.m[0];
    case 1: return &maps.m[1];
    case 2: return &maps.m[2];
    case 3: return &maps.m[3];
    case 4: return &maps.m[4];
    case 5: return &maps.m[5];
    case 6: return &maps.m[6];
    default: return &maps.m[7];
  }
}

struct TtTile {
  int j, z, i0;     // job, product within the job, first row
};

// (jobs: the launch's jobs copied to shared memory: reading the job of a tile straight from
// the kernel parameter at a run-time index gave wrong rows in the library build, and the
// tensor maps are taken at constant offsets for the same reason)
__device__ __forceinline__ TtTile tile_of(const TtJob* jobs, int njob, int tile, int mt) {
  TtTile t;
  t.j = (njob > 1 && tile >= jobs[1].tile0) ? 1 : 0;
  const int local = tile - jobs[t.j].tile0;
  t.z = local / mt;
  t.i0 = (local - t.z * mt) * TT_ROWS;
  return t;
}

// stages of output z of a job and whether each segment takes part
__device__ __forceinline__ int tile_stages(const TtJob& q, int z, bool& v0, bool& v1) {
  v0 = z >= q.seg[0].zlo && z < q.seg[0].zhi;
  v1 = q.nseg > 1 && z >= q.seg[1].zlo && z < q.seg[1].zhi;
  return (v0 ? q.seg[0].nkb : 0) + (v1 ? q.seg[1].nkb : 0);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of real element (n, k) of a K-major, no-swizzle B stage (16 real k)
__device__ __forceinline__ uint32_t bcore_off(int n, int k) {
  return (uint32_t)(n >> 3) * TT_SBO + (uint32_t)(k >> 2) * TT_LBO + (uint32_t)(n & 7) * 16u +
         (uint32_t)(k & 3) * 4u;
}

__device__ __forceinline__ uint64_t bdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((TT_LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((TT_SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle
  return d;
}

// shared-memory address of 16-byte chunk c of row r in a tile of 64-byte rows written by
// TMA with the 64-byte swizzle: the chunk index is XORed with bits 7-8 of the row's address
__device__ __forceinline__ uint32_t sw64_addr(uint32_t tile, int r, int c) {
  const uint32_t row = tile + (uint32_t)r * 64u;
  return row + (((uint32_t)c ^ (row >> 7)) & 3u) * 16u;
}

__device__ __forceinline__ void sts128(uint32_t a, const float (&v)[4]) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]),
               "f"(v[3])
               : "memory");
}

__device__ __forceinline__ float4 lds128(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}

// TF32 hi part rounded to nearest (ties away), lo = x - hi exact (as in tc_gemm.cu)
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  lo = x - hi;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  return done != 0u;
}

// bounded wait that ignores the abort flag (the kernel's own copies and MMAs before exit)
__device__ __forceinline__ bool tt_wait_own(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    if (mbar_test(a, parity)) return true;
    if (clock64() - t0 > TT_DEFAULT_WAIT) return false;
  }
}

// bounded wait taken by the whole warp together (no divergence): the phase has completed
// once any lane sees it complete; the warp gives up together on the abort flag or the limit
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          long long limit) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    if (__any_sync(0xffffffffu, mbar_test(a, parity))) return true;
    const bool expired = clock64() - t0 > limit;
    if (__any_sync(0xffffffffu, expired || *abort_flag != 0)) {
      if (expired) *abort_flag = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_tf32_ta(uint32_t d, uint32_t a_tmem, uint64_t b,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
      : "memory");
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
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__global__ void __launch_bounds__(TT_THREADS, 1)
    tc_cgemm_tma_kernel(const __grid_constant__ TtMaps maps, const __grid_constant__ TtArgs p) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm_raw + TT_BAR_OFF);
  uint64_t* raw_full = bars;
  uint64_t* raw_empty = raw_full + TT_RS;
  uint64_t* conv_full = raw_empty + TT_RS;
  uint64_t* conv_empty = conv_full + TT_CS;
  uint64_t* acc_full = conv_empty + TT_CS;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* done_bar = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = (p.M + TT_ROWS - 1) / TT_ROWS;               // row tiles per product
  const int64_t ntiles = p.ntiles;
  const int ntl = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  const int NB = p.NB;
  // the swizzled TMA destinations assume a 1024-byte aligned shared-memory window: refuse to
  // run (before any copy or allocation) where it is not
  if (smem_u32(sm_raw) & 1023u) {
    if (tid == 0) atomicCAS(p.status, DEV_OK, DEV_BADINPUT);
    return;
  }

  __shared__ TtJob jobs[2];
  if (tid == 0) {
    jobs[0] = p.job[0];
    jobs[1] = p.job[1];
    for (int s = 0; s < TT_RS; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], TT_GWARPS);
    }
    for (int s = 0; s < TT_CS; ++s) {
      mbar_init(&conv_full[s], TT_GWARPS);
      mbar_init(&conv_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == TT_TMA_WARP) {
    // ------------------------------------------------------------ TMA producer
    // (the warp waits together; lane 0 issues the copies)
    {
      const uint32_t bytes = TT_RAW_A + (uint32_t)NB * TT_KC * 8u;
      int it = 0;
      bool ok = true;
      for (int tl = 0; tl < ntl && ok; ++tl) {
        const TtTile t = tile_of(jobs, p.njob, (int)blockIdx.x + tl * (int)gridDim.x, mt);
        const TtJob& q = jobs[t.j];
        bool v0, v1;
        const int nst = tile_stages(q, t.z, v0, v1);
        for (int st = 0; st < nst; ++st, ++it) {
          const int s = it % TT_RS;
          if (it >= TT_RS &&
              !warp_wait(&raw_empty[s], (uint32_t)((it / TT_RS - 1) & 1), abort_flag, p.wait_limit)) {
            ok = false;
            break;
          }
          if (lane != 0) continue;
          const int g = (!v0 || st >= q.seg[0].nkb) ? 1 : 0;
          const TtSeg& sg = q.seg[g];
          const int k0 = (g ? (v0 ? st - q.seg[0].nkb : st) : st) * TT_KC;
          unsigned char* rs = sm_raw + (size_t)s * TT_RAW_STAGE;
          const uint32_t ra = smem_u32(rs), rb = smem_u32(rs + TT_RAW_A);
          const CUtensorMap* mA = map_at(maps, 4 * t.j + 2 * g);
          const CUtensorMap* mB = map_at(maps, 4 * t.j + 2 * g + 1);
          const int za = t.z + sg.zA, zb = t.z + sg.zB;
          mbar_expect_tx(&raw_full[s], bytes);
          if (!sg.ta) tma_load_3d(ra, mA, k0, t.i0, za, &raw_full[s]);
          else tma_load_3d(ra, mA, t.i0, k0, za, &raw_full[s]);
          if (!sg.tb) tma_load_3d(rb, mB, 0, k0, zb, &raw_full[s]);
          else tma_load_3d(rb, mB, k0, 0, zb, &raw_full[s]);
        }
      }
      // the copies lane 0 issued land before the CTA can exit
      if (lane == 0)
        for (int d = it - TT_RS < 0 ? 0 : it - TT_RS; d < it; ++d)
          if (!tt_wait_own(&raw_full[d % TT_RS], (uint32_t)((d / TT_RS) & 1))) *abort_flag = 1;
    }
    __syncwarp();
  } else if (warp < TT_CONV_WARPS) {
    // ------------------------------------------------------------ converters
    const int grp = warp / TT_GWARPS, gw = warp % TT_GWARPS, gtid = tid % TT_GTHREADS;
    const int q = warp & 3;               // tensor-memory lane quarter
    const int kh0 = TT_KSPLIT == 2 ? gw >> 2 : 0;  // first half of the stage's k it converts
    const int l = 16 * q + (lane >> 1);  // complex row of the tile
    const int part = lane & 1;           // 0: (ar, -ai) -> Re rows; 1: (ai, ar) -> Im rows
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    // this thread's B items e = gtid + group size * r: column n, pair j of complex k (2 j,
    // 2 j + 1); packed n | j << 16 (-1: none), the raw-tile read index (op = N) and the
    // offset in the split stage
    int bitem[TT_BITEMS], brd[TT_BITEMS];
    uint32_t boff[TT_BITEMS];
#pragma unroll
    for (int r = 0; r < TT_BITEMS; ++r) {
      const int e = gtid + TT_GTHREADS * r;
      const int j = e / NB, n = e - j * NB;
      const bool v = e < 4 * NB;
      bitem[r] = v ? (n | (j << 16)) : -1;
      brd[r] = (2 * j) * NB + n;
      boff[r] = bcore_off(n, 4 * j);
    }
    int it = 0;
    bool ok = true;
    for (int tl = 0; tl < ntl && ok; ++tl) {
      const TtTile t = tile_of(jobs, p.njob, (int)blockIdx.x + tl * (int)gridDim.x, mt);
      const TtJob& q = jobs[t.j];
      bool v0, v1;
      const int nst = tile_stages(q, t.z, v0, v1);
      for (int st = 0; st < nst; ++st, ++it) {
        if (it % TT_GROUPS != grp) continue;
        const int g = (!v0 || st >= q.seg[0].nkb) ? 1 : 0;
        const bool ta = q.seg[g].ta != 0, tb = q.seg[g].tb != 0;
        const int s = it % TT_RS, cs = it % TT_CS;
        if (!warp_wait(&raw_full[s], (uint32_t)((it / TT_RS) & 1), abort_flag, p.wait_limit)) {
          ok = false;
          break;
        }
        if (it >= TT_CS && !warp_wait(&conv_empty[cs], (uint32_t)((it / TT_CS - 1) & 1), abort_flag,
                                      p.wait_limit)) {
          ok = false;
          break;
        }
        fence_after();
        const unsigned char* rs = sm_raw + (size_t)s * TT_RAW_STAGE;
        // A: four complex k of row l per half of the stage's k
#pragma unroll
        for (int hh = 0; hh < 3 - TT_KSPLIT; ++hh) {
          const int kh = kh0 + hh;
          float2 a[4];
          if (!ta) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const float4 v = lds128(sw64_addr(smem_u32(rs), l, 2 * kh + c));
              a[2 * c] = make_float2(v.x, v.y);
              a[2 * c + 1] = make_float2(v.z, v.w);
            }
          } else {
            const float2* ra = reinterpret_cast<const float2*>(rs);
#pragma unroll
            for (int j = 0; j < 4; ++j) a[j] = ra[(4 * kh + j) * TT_ROWS + l];
          }
          float hi[8], lo[8];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float x0 = part ? a[j].y : a[j].x;
            const float x1 = part ? a[j].x : -a[j].y;
            split_tf32(x0, hi[2 * j], lo[2 * j]);
            split_tf32(x1, hi[2 * j + 1], lo[2 * j + 1]);
          }
          const uint32_t slot = lane_base + a_slot(cs) + 8u * (uint32_t)kh;
          tmem_st8(slot, hi);
          tmem_st8(slot + 16u, lo);
        }
        // B: this thread's (n, j) items, all loads first, then the splits and stores
        const unsigned char* rb = rs + TT_RAW_A;
        const uint32_t rbu = smem_u32(rb);
        const uint32_t bsu = smem_u32(sm_raw + TT_CONV_OFF + (size_t)cs * TT_CSTAGE);
        float4 bv[TT_BITEMS];
#pragma unroll
        for (int r = 0; r < TT_BITEMS; ++r) {
          if (bitem[r] < 0) continue;
          if (!tb) {
            const float2* rbb = reinterpret_cast<const float2*>(rb);
            const float2 b0 = rbb[brd[r]], b1 = rbb[brd[r] + NB];
            bv[r] = make_float4(b0.x, b0.y, b1.x, b1.y);
          } else {
            bv[r] = lds128(sw64_addr(rbu, bitem[r] & 0xFFFF, bitem[r] >> 16));
          }
        }
#pragma unroll
        for (int r = 0; r < TT_BITEMS; ++r) {
          if (bitem[r] < 0) continue;
          float h[4], o[4];
          split_tf32(bv[r].x, h[0], o[0]);
          split_tf32(bv[r].y, h[1], o[1]);
          split_tf32(bv[r].z, h[2], o[2]);
          split_tf32(bv[r].w, h[3], o[3]);
          sts128(bsu + boff[r], h);
          sts128(bsu + TT_BSPLIT + boff[r], o);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&conv_full[cs]);
          mbar_arrive(&raw_empty[s]);
        }
      }
    }
  } else if (warp == TT_MMA_WARP) {
    // ------------------------------------------------------------ MMA issue
    // (the warp waits together; lane 0 issues the MMAs and commits)
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NB >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    bool ok = true;
    int it = 0;
    for (int tl = 0; tl < ntl && ok; ++tl) {
      const int b = tl & 1;
      if (tl >= 2 &&
          !warp_wait(&acc_empty[b], (uint32_t)((tl / 2 - 1) & 1), abort_flag, p.wait_limit))
        break;
      fence_after();
      const uint32_t acc = tmem + (uint32_t)b * TT_ACC_STRIDE;
      const TtTile t = tile_of(jobs, p.njob, (int)blockIdx.x + tl * (int)gridDim.x, mt);
      bool v0, v1;
      const int nst = tile_stages(jobs[t.j], t.z, v0, v1);
      for (int st = 0; st < nst; ++st, ++it) {
        const int cs = it % TT_CS;
        if (!warp_wait(&conv_full[cs], (uint32_t)((it / TT_CS) & 1), abort_flag, p.wait_limit)) {
          ok = false;
          break;
        }
        fence_after();
        if (lane == 0) {
          const uint32_t aslot = tmem + a_slot(cs);
          const uint32_t bh = smem_u32(sm_raw + TT_CONV_OFF + (size_t)cs * TT_CSTAGE);
          const uint32_t bl = bh + TT_BSPLIT;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint32_t boff = (uint32_t)ks * 2u * TT_LBO;
            const uint32_t ah = aslot + 8u * (uint32_t)ks, al = ah + 16u;
            mma_tf32_ta(acc, ah, bdesc(bh + boff), idesc, (st | ks) ? 1u : 0u);
            mma_tf32_ta(acc, ah, bdesc(bl + boff), idesc, 1u);
            mma_tf32_ta(acc, al, bdesc(bh + boff), idesc, 1u);
          }
          mma_commit(&conv_empty[cs]);
        }
        __syncwarp();
      }
      if (ok && lane == 0) mma_commit(&acc_full[b]);
      __syncwarp();
    }
    // every MMA issued by lane 0 has finished before the tensor memory is freed
    if (lane == 0) {
      mma_commit(done_bar);
      if (!tt_wait_own(done_bar, 0)) *abort_flag = 1;
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // a warp may read tensor-memory lanes 32 (warp % 4) .. + 31
    const int l = 16 * q + (lane >> 1);
    const int part = lane & 1;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    const int nch = NB / 16;
    for (int tl = 0; tl < ntl; ++tl) {
      const int b = tl & 1;
      const TtTile t = tile_of(jobs, p.njob, (int)blockIdx.x + tl * (int)gridDim.x, mt);
      const TtJob& qj = jobs[t.j];
      const bool has_c0 = qj.C0 != nullptr && qj.beta != 0.f;
      const float alpha = qj.alpha, beta = qj.beta;
      const int z = t.z;
      const int row = t.i0 + l;
      const bool rok = row < p.M;
      float2* Crow = qj.C + (int64_t)z * qj.sC + (int64_t)(rok ? row : 0) * qj.ldc;
      const float2* C0row =
          has_c0 ? qj.C0 + (int64_t)z * qj.sC0 + (int64_t)(rok ? row : 0) * qj.ldc0 : nullptr;
      // C0 of chunk c: four 16-byte pieces, columns 16 c + 4 j + 2 part (+1)
      auto load_c0 = [&](int c, float4 (&dst)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int col = 16 * c + 4 * j + 2 * part;
          dst[j] = (has_c0 && rok && col < p.N)
                       ? *reinterpret_cast<const float4*>(C0row + col)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      };
      float4 c0a[4], c0b[4];
      load_c0(0, c0a);
      if (!warp_wait(&acc_full[b], (uint32_t)((tl / 2) & 1), abort_flag, p.wait_limit)) break;
      fence_after();
      bool v0, v1;
      const bool empty = tile_stages(qj, z, v0, v1) == 0;  // no MMA: the product is zero
      for (int c = 0; c < nch; ++c) {
        float v[16];
        tmem_ld16(lane_base + (uint32_t)b * TT_ACC_STRIDE + 16u * (uint32_t)c, v);
        if (empty) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
        if (c == nch - 1) {
          // the accumulator has been read: the next tile's MMAs may overwrite it
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        if (c + 1 < nch) load_c0(c + 1, c0b);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // even lane: Re of columns 4 j, 4 j + 1 (its own) + Im from the odd lane;
          // odd lane: Im of columns 4 j + 2, 4 j + 3 (its own) + Re from the even lane
          const float s0 = part ? v[4 * j] : v[4 * j + 2];
          const float s1 = part ? v[4 * j + 1] : v[4 * j + 3];
          const float r0 = __shfl_xor_sync(0xffffffffu, s0, 1);
          const float r1 = __shfl_xor_sync(0xffffffffu, s1, 1);
          float4 o = part ? make_float4(r0, v[4 * j + 2], r1, v[4 * j + 3])
                          : make_float4(v[4 * j], r0, v[4 * j + 1], r1);
          const int col = 16 * c + 4 * j + 2 * part;
          if (rok && col < p.N) {
            o.x *= alpha;
            o.y *= alpha;
            o.z *= alpha;
            o.w *= alpha;
            if (has_c0) {
              o.x = fmaf(beta, c0a[j].x, o.x);
              o.y = fmaf(beta, c0a[j].y, o.y);
              o.z = fmaf(beta, c0a[j].z, o.z);
              o.w = fmaf(beta, c0a[j].w, o.w);
            }
            *reinterpret_cast<float4*>(Crow + col) = o;
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) c0a[j] = c0b[j];
      }
    }
  }
  fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicCAS(p.status, DEV_OK, DEV_TIMEOUT);
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TT_TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- host side
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

// 3-d map over complex64 elements (as 8-byte words): inner extent d0 (contiguous), d1 rows
// `ld` elements apart, d2 batch members `sb` elements apart; box b0 x b1 x 1
bool make_map(CUtensorMap* m, const float2* base, uint64_t d0, uint64_t d1, uint64_t d2,
              int64_t ld, int64_t sb, uint32_t b0, uint32_t b1, bool sw64) {
  EncodeTiled enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * 8u, (cuuint64_t)sb * 8u};
  const cuuint32_t box[3] = {b0, b1, 1u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2*>(base), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             sw64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 1;
    return v > 0 ? v : 1;
  }();
  return n;
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

namespace {

// tensor maps of one segment's operands; false where TMA cannot take them
bool seg_maps(const TcSegment& g, int M, int N, int NB, CUtensorMap* mA, CUtensorMap* mB) {
  if (g.K < 1 || g.nA < 1 || g.nB < 1 || !al16(g.A) || !al16(g.B) || ((g.lda | g.ldb) & 1))
    return false;
  if ((g.nA > 1 && (g.sA <= 0 || (g.sA & 1))) || (g.nB > 1 && (g.sB <= 0 || (g.sB & 1))))
    return false;
  // a single member: any stride the map accepts
  const int64_t sa = g.nA > 1 ? g.sA : g.lda * (g.ta ? g.K : M);
  const int64_t sb = g.nB > 1 ? g.sB : g.ldb * (g.tb ? N : g.K);
  // A: op = N stored [M][K] (64-byte rows, swizzled); op = T stored [K][M]
  const bool okA = !g.ta ? make_map(mA, g.A, (uint64_t)g.K, (uint64_t)M, (uint64_t)g.nA, g.lda, sa,
                                    TT_KC, TT_ROWS, true)
                         : make_map(mA, g.A, (uint64_t)M, (uint64_t)g.K, (uint64_t)g.nA, g.lda, sa,
                                    TT_ROWS, TT_KC, false);
  // B: op = N stored [K][N]; op = T stored [N][K] (64-byte rows, swizzled)
  const bool okB = !g.tb ? make_map(mB, g.B, (uint64_t)N, (uint64_t)g.K, (uint64_t)g.nB, g.ldb, sb,
                                    (uint32_t)NB, TT_KC, false)
                         : make_map(mB, g.B, (uint64_t)g.K, (uint64_t)N, (uint64_t)g.nB, g.ldb, sb,
                                    TT_KC, (uint32_t)NB, true);
  return okA && okB;
}

}  // namespace

cudaError_t launch_tc_cgemm_tma_jobs(int M, int N, int njob, const TcJob* jobs, int32_t* status,
                                     long long wait_limit, cudaStream_t s) {
  // the shapes and alignments the TMA boxes and the 16-byte epilogue stores need
  if (M < 1 || N < 2 || N > TT_NMAX || (N & 1) || njob < 1 || njob > 2)
    return cudaErrorNotSupported;
  const int NB = (N + 15) & ~15;
  const int mt = (M + TT_ROWS - 1) / TT_ROWS;
  TtMaps maps{};
  TtArgs a{};
  a.M = M;
  a.N = N;
  a.NB = NB;
  a.status = status;
  a.wait_limit = wait_limit;
  int64_t ntiles = 0;
  for (int jb = 0; jb < njob; ++jb) {
    const TcJob& jo = jobs[jb];
    if (jo.batch <= 0) continue;  // an empty job takes no tiles
    if (jo.batch > 65535 || jo.nseg < 1 || jo.nseg > 2) return cudaErrorNotSupported;
    if (!al16(jo.C) || (jo.ldc & 1) || (jo.C0 && (!al16(jo.C0) || (jo.ldc0 & 1))))
      return cudaErrorNotSupported;
    TtJob& q = a.job[a.njob];
    for (int g = 0; g < jo.nseg; ++g) {
      const TcSegment& sg = jo.seg[g];
      CUtensorMap* mA = &maps.m[4 * a.njob + 2 * g];
      if (!seg_maps(sg, M, N, NB, mA, mA + 1)) return cudaErrorNotSupported;
      // the members each output reads must exist
      const int lo = sg.zlo < 0 ? 0 : sg.zlo, hi = sg.zhi > jo.batch ? jo.batch : sg.zhi;
      if (hi > lo && (lo + sg.zA < 0 || hi - 1 + sg.zA >= sg.nA || lo + sg.zB < 0 ||
                      hi - 1 + sg.zB >= sg.nB))
        return cudaErrorNotSupported;
      q.seg[g] = TtSeg{(sg.K + TT_KC - 1) / TT_KC, sg.zA, sg.zB, lo, hi, sg.ta ? 1 : 0,
                       sg.tb ? 1 : 0};
    }
    q.batch = jo.batch;
    q.nseg = jo.nseg;
    q.tile0 = (int)ntiles;
    q.C = jo.C;
    q.ldc = jo.ldc;
    q.sC = jo.sC;
    q.C0 = jo.C0;
    q.ldc0 = jo.ldc0;
    q.sC0 = jo.sC0;
    q.alpha = jo.alpha;
    q.beta = jo.beta;
    ntiles += (int64_t)jo.batch * mt;
    ++a.njob;
  }
  if (a.njob == 0) return cudaSuccess;
  a.ntiles = (int)ntiles;
  const unsigned grid = (unsigned)(ntiles < sms() ? ntiles : sms());
  RCI_CUDA_TRY(cudaFuncSetAttribute(tc_cgemm_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)TT_SMEM));
  tc_cgemm_tma_kernel<<<grid, TT_THREADS, TT_SMEM, s>>>(maps, a);
  rci_note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_cgemm_tma_seg(int M, int N, int nseg, const TcSegment* seg, float alpha,
                                    float beta, const float2* C0, int64_t ldc0, int64_t sC0,
                                    float2* C, int64_t ldc, int64_t sC, int batch, int32_t* status,
                                    long long wait_limit, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  if (nseg < 1 || nseg > 2) return cudaErrorNotSupported;
  TcJob jo{};
  jo.nseg = nseg;
  for (int g = 0; g < nseg; ++g) jo.seg[g] = seg[g];
  jo.alpha = alpha;
  jo.beta = beta;
  jo.C0 = C0;
  jo.ldc0 = ldc0;
  jo.sC0 = sC0;
  jo.C = C;
  jo.ldc = ldc;
  jo.sC = sC;
  jo.batch = batch;
  return launch_tc_cgemm_tma_jobs(M, N, 1, &jo, status, wait_limit, s);
}

cudaError_t launch_tc_cgemm_tma(int M, int N, int K, bool ta, bool tb, float alpha,
                                const float2* A, int64_t lda, int64_t sA, const float2* B,
                                int64_t ldb, int64_t sB, float beta, const float2* C0,
                                int64_t ldc0, int64_t sC0, float2* C, int64_t ldc, int64_t sC,
                                int batch, int32_t* status, long long wait_limit, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  if (K < 1) return cudaErrorNotSupported;
  TcSegment g{A, lda, sA, batch, ta, B, ldb, sB, batch, tb, K, 0, 0, 0, batch};
  return launch_tc_cgemm_tma_seg(M, N, 1, &g, alpha, beta, C0, ldc0, sC0, C, ldc, sC, batch,
                                 status, wait_limit, s);
}
