// Batched complex FP32 GEMM on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
//   C[z] = alpha op(A[z]) op(B[z]) + beta C0[z]      (row-major, op = N or T, complex)
//
// Complex product as one real product: with interleaved storage a complex M x K matrix
// A is already the real M x 2K matrix [re im re im ...]; B is expanded per element into
// the 2 x 2 real block [[br, bi], [-bi, br]], so the real product's 2N accumulator
// columns are the interleaved real and imaginary parts of C.
//
// FP32 accuracy from TF32 inputs ("3xTF32"): every operand x is split into x_hi =
// tf32(x) (round to nearest) and x_lo = x - x_hi, and the accumulator takes
// A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 (the missing A_lo B_lo term is ~2^-22
// relative).  The solver's FP64 iterative refinement absorbs the rest.
//
// Three kernels.  For real alpha and beta, even N <= 160 and 16-byte aligned operands
// (every product of the block solver) the TMA-fed kernel of tc_gemm_tma.cu, with the A
// operand in tensor memory.  Where its alignment rules fail, the persistent stacked form
// below: one CTA per SM, warp-specialised (register-staged operands, MMA issue, epilogue),
// 128-row tiles of the stacked product, accumulators double buffered in tensor memory.
// Otherwise (complex scalars, larger N) the expanded-B form: one CTA per 128 x 80 complex
// output tile (M = 128 rows, N = 160 real columns per MMA); K in chunks of 8 complex (16
// real) per pipeline stage, 3 stages (two CTAs per SM).  All 256 threads stage operands
// (global -> registers, issued ahead -> split -> shared memory in the K-major, no-swizzle
// core-matrix layout); thread 0 issues the MMAs for a stage and commits them to that
// stage's mbarrier, which releases the buffer for reuse.  The accumulator lives in tensor
// memory (160 of 256 allocated columns) and is read back by the 8 warps (warp w: lanes
// 32 (w % 4).., columns half (w / 4)).
// Every wait is bounded: on timeout the kernel records DEV_TIMEOUT in *status, skips
// the epilogue, frees its tensor memory and returns.
#include <atomic>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int TC_THREADS = 256;
constexpr int TM = 128;          // output rows per CTA (UMMA M)
constexpr int TNC = 80;          // complex output columns per CTA
constexpr int TNR = 2 * TNC;     // real accumulator columns (UMMA N)
constexpr int KC = 8;            // complex k per stage
constexpr int KR = 2 * KC;       // real k per stage
constexpr int NSTAGE = 3;
constexpr int TMEM_COLS = 256;
constexpr uint32_t CORE_BYTES = 128;             // 8 rows x 16 bytes
constexpr uint32_t LBO = CORE_BYTES;             // next core matrix along K
constexpr uint32_t SBO = (KR / 4) * CORE_BYTES;  // next 8-row group
constexpr uint32_t A_BYTES = TM * KR * 4;        // one split of the A tile
constexpr uint32_t B_BYTES = TNR * KR * 4;       // one split of the B tile
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr size_t SMEM_BYTES = (size_t)NSTAGE * STAGE_BYTES + 1024;
constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz
constexpr int EP_LD = TNR + 1;                   // epilogue tile row stride (floats)
static_assert((size_t)TM * EP_LD * 4 <= (size_t)NSTAGE * STAGE_BYTES,
              "the epilogue tile reuses the stage buffers");

struct TcArgs {
  int M, N, K;
  const float2* A;
  int64_t lda, sA;
  const float2* B;
  int64_t ldb, sB;
  float2* C;
  int64_t ldc, sC;
  const float2* C0;
  int64_t ldc0, sC0;
  float2 alpha, beta;
  int32_t* status;
  int batch;
  long long wait_limit;  // SM clock cycles a pipeline wait may take before the kernel gives up
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of real element (r, k) of a K-major no-swizzle tile with KR real k
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)(r >> 3) * SBO + (uint32_t)(k >> 2) * LBO + (uint32_t)(r & 7) * 16u +
         (uint32_t)(k & 3) * 4u;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle (layout type 0)
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, N = TNR, M = TM
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TNR >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

// x_hi = x rounded to TF32 (10 mantissa bits), to nearest with ties away from zero: half a
// TF32 unit (bit 12) added to the magnitude bits, then the 13 low bits cleared (a carry into
// the exponent is the correct rounding up to the next binade); x_lo = x - x_hi is exact.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  lo = x - hi;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// true when the phase with the given parity has completed; false after `limit` cycles
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = WAIT_LIMIT_CYCLES) {
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

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 consecutive columns as two x16 loads and one wait
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[16], float (&w)[16]) {
  uint32_t r[16], q[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]),
        "=r"(q[7]), "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]),
        "=r"(q[14]), "=r"(q[15])
      : "r"(taddr + 16u));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v[i] = __uint_as_float(r[i]);
    w[i] = __uint_as_float(q[i]);
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
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(TC_THREADS, 2) tc_cgemm_kernel(TcArgs p) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  // stage buffers, then the mbarriers and the tensor-memory address slot
  unsigned char* stages = sm_raw;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm_raw + (size_t)NSTAGE * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + NSTAGE);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t z = blockIdx.z;
  const float2* A = p.A + z * p.sA;
  const float2* B = p.B + z * p.sB;
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TNC;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(&mbar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nkb = (p.K + KC - 1) / KC;
  // Work items are pairs of consecutive complex k (= one 16-byte core-matrix row of four
  // real k), so every shared-memory store is a full 16-byte row.
  //   A: 128 rows x 4 pairs = 512 items, 2 per thread (row am[q], pair apa[q]);
  //   B: 80 columns x 4 pairs = 320 items, up to 2 per thread (column bn[r], pair bpb[r]).
  int am[2], apa[2], bn[2], bpb[2];
  bool bval[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (!TA) {
      const int e = tid * 2 + q;  // two consecutive pairs (4 consecutive k) of one row
      am[q] = e >> 2;
      apa[q] = e & 3;
    } else {
      const int e = tid + TC_THREADS * q;  // consecutive rows across a warp
      am[q] = e & (TM - 1);
      apa[q] = e >> 7;
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int e = tid + TC_THREADS * r;
    bval[r] = e < TNC * (KC / 2);
    if (!TB) {
      bn[r] = e % TNC;  // consecutive columns across a warp
      bpb[r] = e / TNC;
    } else {
      bpb[r] = e & 3;  // consecutive k pairs of one column
      bn[r] = e >> 2;
    }
  }
  auto load_stage = [&](int kb, float2 (&av)[2][2], float2 (&bv)[2][2]) {
    const int k0 = kb * KC;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int gi = i0 + am[q], gk = k0 + 2 * apa[q] + c;
        av[q][c] = make_float2(0.f, 0.f);
        if (gi < p.M && gk < p.K)
          av[q][c] = TA ? A[(int64_t)gk * p.lda + gi] : A[(int64_t)gi * p.lda + gk];
      }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int gk = k0 + 2 * bpb[r] + c, gj = j0 + bn[r];
        bv[r][c] = make_float2(0.f, 0.f);
        if (bval[r] && gk < p.K && gj < p.N)
          bv[r][c] = TB ? B[(int64_t)gj * p.ldb + gk] : B[(int64_t)gk * p.ldb + gj];
      }
  };
  // Operand loads run PF stages ahead through a ring of register sets (static indices: the
  // K loop is unrolled by the ring length), so their latency overlaps PF stages of work.
  constexpr int PF = 3, RING = PF + 1;
  float2 av[RING][2][2], bv[RING][2][2];
#pragma unroll
  for (int d = 0; d < PF; ++d)
    if (d < nkb) load_stage(d, av[d], bv[d]);
  bool ok = true;
  int committed = -1;  // last stage whose MMAs thread 0 committed (uniform across the CTA)
  for (int base = 0; base < nkb && ok; base += RING) {
#pragma unroll
    for (int g = 0; g < RING; ++g) {
      const int kb = base + g;
      if (kb >= nkb || !ok) break;
      const int st = kb % NSTAGE;
      unsigned char* sb = stages + (size_t)st * STAGE_BYTES;
      if (kb + PF < nkb) load_stage(kb + PF, av[(g + PF) % RING], bv[(g + PF) % RING]);
      if (kb >= NSTAGE) {
        // the MMAs that last read this buffer must have completed
        if (!mbar_wait(&mbar[st], (uint32_t)((kb / NSTAGE - 1) & 1), p.wait_limit)) ok = false;
      }
      if (__syncthreads_or(!ok)) {
        ok = false;
        break;
      }
      unsigned char* a_hi = sb;
      unsigned char* a_lo = sb + A_BYTES;
      unsigned char* b_hi = sb + 2 * A_BYTES;
      unsigned char* b_lo = sb + 2 * A_BYTES + B_BYTES;
      // ---- A tile: rows i0 .. i0+127, complex k0 .. k0+7: row am, real k 4 apa .. 4 apa + 3
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float h[4], l[4];
        split_tf32(av[g][q][0].x, h[0], l[0]);
        split_tf32(av[g][q][0].y, h[1], l[1]);
        split_tf32(av[g][q][1].x, h[2], l[2]);
        split_tf32(av[g][q][1].y, h[3], l[3]);
        const uint32_t o = core_off(am[q], 4 * apa[q]);
        *reinterpret_cast<float4*>(a_hi + o) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(a_lo + o) = make_float4(l[0], l[1], l[2], l[3]);
      }
      // ---- B tile: complex k0 .. k0+7, complex columns j0 .. j0+79.  Each complex b
      // expands into the real block [[br, bi], [-bi, br]] at (k', n') = (2k.., 2n..), stored
      // K-major (element (n', k')): row 2n gets (br, -bi), row 2n+1 gets (bi, br) per k.
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!bval[r]) continue;
        float rh0, rl0, ih0, il0, rh1, rl1, ih1, il1;
        split_tf32(bv[g][r][0].x, rh0, rl0);
        split_tf32(bv[g][r][0].y, ih0, il0);
        split_tf32(bv[g][r][1].x, rh1, rl1);
        split_tf32(bv[g][r][1].y, ih1, il1);
        const uint32_t o = core_off(2 * bn[r], 4 * bpb[r]);
        *reinterpret_cast<float4*>(b_hi + o) = make_float4(rh0, -ih0, rh1, -ih1);
        *reinterpret_cast<float4*>(b_hi + o + 16u) = make_float4(ih0, rh0, ih1, rh1);
        *reinterpret_cast<float4*>(b_lo + o) = make_float4(rl0, -il0, rl1, -il1);
        *reinterpret_cast<float4*>(b_lo + o + 16u) = make_float4(il0, rl0, il1, rl1);
      }
      // make the generic-proxy shared-memory writes visible to the tensor cores
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo);
        const uint32_t bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
        for (int ks = 0; ks < KR / 8; ++ks) {
          const uint32_t off = (uint32_t)ks * 2 * LBO;  // 8 real k = two core matrices
          mma_tf32(tmem, smem_desc(ah + off), smem_desc(bh + off), (kb | ks) ? 1u : 0u);
          mma_tf32(tmem, smem_desc(ah + off), smem_desc(bl + off), 1u);
          mma_tf32(tmem, smem_desc(al + off), smem_desc(bh + off), 1u);
        }
        mma_commit(&mbar[st]);
      }
      committed = kb;
    }
  }
  // ---- all committed MMAs done (also after a timeout, before the tensor memory is freed);
  // a commit tracks every earlier MMA of the issuing thread
  if (committed >= 0) {
    if (!mbar_wait(&mbar[committed % NSTAGE], (uint32_t)((committed / NSTAGE) & 1))) ok = false;
  }
  if (committed != nkb - 1) ok = false;
  ok = !__syncthreads_or(!ok);
  if (!ok) {
    if (tid == 0) atomicCAS(p.status, DEV_OK, DEV_TIMEOUT);
  } else {
    // Epilogue through shared memory (the stage buffers are free once every MMA is done):
    // warp w copies TMEM lanes 32 (w % 4).. (tile rows), column half w / 4, into a
    // row-major tile padded to EP_LD floats per row, so both this copy (a row per lane) and
    // the read below (consecutive columns per lane) are free of bank conflicts; then each
    // warp combines and stores rows of C with consecutive complex columns across lanes.
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float* tile = reinterpret_cast<float*>(stages);
    const int lane = tid & 31;
    const int lane_base = 32 * (warp & 3);
    const int col_half = warp >> 2;  // real columns [80 col_half, 80 col_half + 80)
    const int row = lane_base + lane;
#pragma unroll
    for (int c = 0; c < TNR / 2 / 16; ++c) {
      const int col = col_half * (TNR / 2) + 16 * c;
      float v[16];
      tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)col, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) tile[row * EP_LD + col + q] = v[q];
    }
    __syncthreads();
    float2* C = p.C + z * p.sC;
    const float2* C0 = p.C0 ? p.C0 + z * p.sC0 : nullptr;
    for (int r = warp; r < TM; r += TC_THREADS / 32) {
      const int gi = i0 + r;
      if (gi >= p.M) break;
      for (int q = lane; q < TNC; q += 32) {
        const int gj = j0 + q;
        if (gj >= p.N) break;
        const float2 acc = make_float2(tile[r * EP_LD + 2 * q], tile[r * EP_LD + 2 * q + 1]);
        float2 res = p.alpha * acc;
        if (C0) res = cfma(p.beta, C0[(int64_t)gi * p.ldc0 + gj], res);
        C[(int64_t)gi * p.ldc + gj] = res;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- stacked form
// For real alpha and beta, the complex product as the real product of the stacked
//   A_s = [[Ar, -Ai], [Ai, Ar]]  (2M x 2K: the pairs (ar, -ai) per complex k on the rows of
//   the top half, (ai, ar) on the bottom half)   and   B_s = [Br; Bi]  (2K x N, (br, bi) per k),
// so C_s = A_s B_s holds Re C in its first M rows and Im C in the next M.  One 128-row tile
// of C_s covers 160 complex columns, and 2M = 320 rows fill three tiles where the
// expanded-B form needs four 128 x 80 tiles for a 160 x 160 product; B is staged as it is
// stored (one 16-byte core row per pair of complex k instead of two).
constexpr int TNS = 160;                          // complex (= real) columns per CTA
constexpr uint32_t BS_BYTES = TNS * KR * 4;       // one split of the B_s tile
constexpr uint32_t SSTAGE_BYTES = 2 * A_BYTES + 2 * BS_BYTES;
constexpr uint32_t IDESC_S = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TNS >> 3) << 17) |
                             ((uint32_t)(TM >> 4) << 24);
constexpr int SB_ITEMS = (TNS * (KC / 2) + TC_THREADS - 1) / TC_THREADS;  // 3

__device__ __forceinline__ void mma_tf32_s(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC_S), "r"(accumulate));
}

// ---------------------------------------------------------------- persistent stacked form
// The stacked product with the roles of a CTA split, one CTA per SM looping over the
// 128-row tiles (tile = product z x row tile y, CTA b takes tiles b, b + grid, ...):
//   warps 0-7   stage operands: global -> registers (two stages ahead) -> TF32 hi/lo ->
//               a ring of WS_NSTAGE shared-memory stages; each warp arrives once on the
//               stage's "full" barrier, and waits on its "empty" barrier before reuse;
//   warp 12     (one lane) waits "full", issues the six MMAs of a stage and commits them
//               to "empty"; after a tile's last stage it commits to "acc full";
//   warps 8-11  wait "acc full", read the accumulator from tensor memory in 32-column
//               chunks (warp 8 + w reads lanes 32 w ..), release it ("acc empty") and
//               write C through a private padded shared-memory slice per warp, with
//               stores along the rows of C.
// Two accumulators (tensor-memory columns 0 and 256) let the epilogue of one tile run
// under the MMAs of the next.  Every wait is bounded; the first that runs out sets a
// shared abort flag that ends the other roles' waits, the kernel records DEV_TIMEOUT,
// waits (bounded) for its own MMAs to finish, frees its tensor memory and returns.
constexpr int WS_PROD_WARPS = 8, WS_EPI_WARP0 = 8, WS_MMA_WARP = 12;
constexpr int WS_THREADS = 13 * 32;
constexpr int WS_NSTAGE = 4;
constexpr int WS_EPI_CH = 32;                    // accumulator columns per epilogue chunk
constexpr int WS_EPI_LD = WS_EPI_CH + 1;
constexpr uint32_t WS_TMEM_COLS = 512;
constexpr uint32_t WS_ACC_STRIDE = 256;
constexpr size_t WS_EPI_OFF = (size_t)WS_NSTAGE * SSTAGE_BYTES;
constexpr size_t WS_BAR_OFF = WS_EPI_OFF + (size_t)TM * WS_EPI_LD * 4;
constexpr size_t WS_SMEM_BYTES = WS_BAR_OFF + 256;
static_assert(WS_PROD_WARPS * 32 == TC_THREADS, "the staging map assumes 256 threads");
static_assert(TNS % WS_EPI_CH == 0, "whole epilogue chunks");

// bounded wait that also ends when another role has given up
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                        long long limit) {
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
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar))
      : "memory");
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(WS_THREADS, 1) tc_cgemm_ws_kernel(TcArgs p) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  unsigned char* stages = sm_raw;
  float* epi = reinterpret_cast<float*>(sm_raw + WS_EPI_OFF);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm_raw + WS_BAR_OFF);
  uint64_t* empty = full + WS_NSTAGE;
  uint64_t* accfull = empty + WS_NSTAGE;
  uint64_t* accempty = accfull + 2;
  uint64_t* done_bar = accempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = (2 * p.M + TM - 1) / TM;                    // row tiles per product
  const int64_t ntiles = (int64_t)mt * p.batch;
  const int ntl = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);  // this CTA's
  const int nkb = (p.K + KC - 1) / KC;

  if (tid == 0) {
    for (int s = 0; s < WS_NSTAGE; ++s) {
      mbar_init(&full[s], WS_PROD_WARPS);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 32 * 4);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(WS_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp < WS_PROD_WARPS) {
    // ------------------------------------------------------------ producers
    int am[2], apa[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!TA) {
        const int e = tid * 2 + q;
        am[q] = e >> 2;
        apa[q] = e & 3;
      } else {
        const int e = tid + TC_THREADS * q;
        am[q] = e & (TM - 1);
        apa[q] = e >> 7;
      }
    }
    int bn[SB_ITEMS], bpb[SB_ITEMS];
    bool bval[SB_ITEMS];
#pragma unroll
    for (int r = 0; r < SB_ITEMS; ++r) {
      const int e = tid + TC_THREADS * r;
      bval[r] = e < TNS * (KC / 2);
      if (!TB) {
        bn[r] = e % TNS;
        bpb[r] = e / TNS;
      } else {
        bpb[r] = e & 3;
        bn[r] = e >> 2;
      }
    }
    // Two cursors over this CTA's stages (tile tl of its list, K block kb): one for the
    // loads, PF stages ahead, one for the stores.  Row and column pointers and the row
    // tests change once per tile; only the last K block of a tile tests k against K.
    struct Cursor {
      int tl, kb, R0;
      const float2* A;
      const float2* B;
    };
    auto set_tile = [&](Cursor& c) {
      const int tile = (int)blockIdx.x + c.tl * (int)gridDim.x;
      const int z = tile / mt;
      c.R0 = (tile - z * mt) * TM;
      c.A = p.A + (int64_t)z * p.sA;
      c.B = p.B + (int64_t)z * p.sB;
    };
    auto advance = [&](Cursor& c) {
      if (++c.kb == nkb) {
        c.kb = 0;
        ++c.tl;
        if (c.tl < ntl) set_tile(c);
      }
    };
    // B columns of this thread (fixed), the A rows of the current load tile
    bool bok[SB_ITEMS];
#pragma unroll
    for (int r = 0; r < SB_ITEMS; ++r) bok[r] = bval[r] && bn[r] < p.N;
    const float2* arow[2];
    bool aok[2];
    int loaded_tl = -1;
    auto load_stage = [&](Cursor& c, float2 (&av)[2][2], float2 (&bv)[SB_ITEMS][2]) {
      if (c.tl != loaded_tl) {
        loaded_tl = c.tl;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int R = c.R0 + am[q];
          const int ar = R < p.M ? R : R - p.M;
          aok[q] = R < 2 * p.M;
          arow[q] = TA ? c.A + ar : c.A + (int64_t)ar * p.lda;
        }
      }
      const int k0 = c.kb * KC;
      const bool kfull = k0 + KC <= p.K;
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int gk = k0 + 2 * apa[q] + cc;
          av[q][cc] = make_float2(0.f, 0.f);
          if (aok[q] && (kfull || gk < p.K))
            av[q][cc] = TA ? arow[q][(int64_t)gk * p.lda] : arow[q][gk];
        }
#pragma unroll
      for (int r = 0; r < SB_ITEMS; ++r)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int gk = k0 + 2 * bpb[r] + cc;
          bv[r][cc] = make_float2(0.f, 0.f);
          if (bok[r] && (kfull || gk < p.K))
            bv[r][cc] = TB ? c.B[(int64_t)bn[r] * p.ldb + gk] : c.B[(int64_t)gk * p.ldb + bn[r]];
        }
      advance(c);
    };
    const int total = ntl * nkb;
    constexpr int PF = 2, RING = PF + 1;
    float2 av[RING][2][2], bv[RING][SB_ITEMS][2];
    Cursor lc{0, 0, 0, nullptr, nullptr}, sc{0, 0, 0, nullptr, nullptr};
    set_tile(lc);
    set_tile(sc);
#pragma unroll
    for (int d = 0; d < PF; ++d)
      if (d < total) load_stage(lc, av[d], bv[d]);
    bool ok = true;
    for (int base = 0; base < total && ok; base += RING) {
#pragma unroll
      for (int g = 0; g < RING; ++g) {
        const int it = base + g;
        if (it >= total) break;
        const int st = it % WS_NSTAGE;
        if (it + PF < total) load_stage(lc, av[(g + PF) % RING], bv[(g + PF) % RING]);
        if (it >= WS_NSTAGE) {
          // one lane per warp polls the barrier
          bool got = true;
          if (lane == 0)
            got = ws_wait(&empty[st], (uint32_t)((it / WS_NSTAGE - 1) & 1), abort_flag, p.wait_limit);
          if (!__shfl_sync(0xffffffffu, got, 0)) {
            ok = false;
            break;
          }
        }
        const int R0 = sc.R0;
        advance(sc);
        unsigned char* sb = stages + (size_t)st * SSTAGE_BYTES;
        unsigned char* a_hi = sb;
        unsigned char* a_lo = sb + A_BYTES;
        unsigned char* b_hi = sb + 2 * A_BYTES;
        unsigned char* b_lo = sb + 2 * A_BYTES + BS_BYTES;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const bool atop = R0 + am[q] < p.M;
          const float2 a0 = av[g][q][0], a1 = av[g][q][1];
          // top half: (ar, -ai) per complex k; bottom half: (ai, ar)
          const float x0 = atop ? a0.x : a0.y, x1 = atop ? -a0.y : a0.x;
          const float x2 = atop ? a1.x : a1.y, x3 = atop ? -a1.y : a1.x;
          float h[4], l[4];
          split_tf32(x0, h[0], l[0]);
          split_tf32(x1, h[1], l[1]);
          split_tf32(x2, h[2], l[2]);
          split_tf32(x3, h[3], l[3]);
          const uint32_t o = core_off(am[q], 4 * apa[q]);
          *reinterpret_cast<float4*>(a_hi + o) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(a_lo + o) = make_float4(l[0], l[1], l[2], l[3]);
        }
#pragma unroll
        for (int r = 0; r < SB_ITEMS; ++r) {
          if (!bval[r]) continue;
          float h[4], l[4];
          split_tf32(bv[g][r][0].x, h[0], l[0]);
          split_tf32(bv[g][r][0].y, h[1], l[1]);
          split_tf32(bv[g][r][1].x, h[2], l[2]);
          split_tf32(bv[g][r][1].y, h[3], l[3]);
          const uint32_t o = core_off(bn[r], 4 * bpb[r]);
          *reinterpret_cast<float4*>(b_hi + o) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(b_lo + o) = make_float4(l[0], l[1], l[2], l[3]);
        }
        // the warp's stores, made visible to the tensor cores, then one arrival per warp
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[st]);
      }
    }
  } else if (warp == WS_MMA_WARP) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      bool ok = true;
      int it = 0;
      for (int tl = 0; tl < ntl && ok; ++tl) {
        const int b = tl & 1;
        if (tl >= 2 &&
            !ws_wait(&accempty[b], (uint32_t)((tl / 2 - 1) & 1), abort_flag, p.wait_limit))
          break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)b * WS_ACC_STRIDE;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int st = it % WS_NSTAGE;
          if (!ws_wait(&full[st], (uint32_t)((it / WS_NSTAGE) & 1), abort_flag, p.wait_limit)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          unsigned char* sb = stages + (size_t)st * SSTAGE_BYTES;
          const uint32_t ah = smem_u32(sb), al = ah + A_BYTES;
          const uint32_t bh = ah + 2 * A_BYTES, bl = bh + BS_BYTES;
#pragma unroll
          for (int ks = 0; ks < KR / 8; ++ks) {
            const uint32_t off = (uint32_t)ks * 2 * LBO;
            mma_tf32_s(acc, smem_desc(ah + off), smem_desc(bh + off), (kb | ks) ? 1u : 0u);
            mma_tf32_s(acc, smem_desc(ah + off), smem_desc(bl + off), 1u);
            mma_tf32_s(acc, smem_desc(al + off), smem_desc(bh + off), 1u);
          }
          mma_commit(&empty[st]);
        }
        if (ok) mma_commit(&accfull[b]);
      }
      // every MMA issued by this thread has finished before the tensor memory is freed
      mma_commit(done_bar);
      if (!mbar_wait(done_bar, 0)) *abort_flag = 1;
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    // warp 8 + w owns tensor-memory lanes 32 w .. 32 w + 31 (rows of the tile) and a
    // private 32 x 33 shared-memory slice in which it turns each 32 x 32 chunk around, so
    // that its stores run along the columns of C
    const int ew = warp - WS_EPI_WARP0;
    float* wt = epi + ew * 32 * WS_EPI_LD;
    for (int tl = 0; tl < ntl; ++tl) {
      const int b = tl & 1;
      // lane 0 polls and the warp follows its verdict: tcgen05.ld below is .sync.aligned,
      // so the whole warp must either go on to it or leave together
      bool got = true;
      if (lane == 0) got = ws_wait(&accfull[b], (uint32_t)((tl / 2) & 1), abort_flag, p.wait_limit);
      if (!__shfl_sync(0xffffffffu, got, 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int tile = (int)blockIdx.x + tl * (int)gridDim.x;
      const int z = tile / mt;
      const int Rw = (tile - z * mt) * TM + 32 * ew;           // first row of this warp
      const bool uniform = Rw + 32 <= p.M || Rw >= p.M;
      const int gi0 = Rw < p.M ? Rw : Rw - p.M, comp0 = Rw < p.M ? 0 : 1;
      const int nval = 2 * p.M - Rw;                           // rows of C_s left (<= 0: none)
      float* C = reinterpret_cast<float*>(p.C + (int64_t)z * p.sC);
      const float* C0 = p.C0 ? reinterpret_cast<const float*>(p.C0 + (int64_t)z * p.sC0) : nullptr;
      for (int c = 0; c < TNS / WS_EPI_CH; ++c) {
        float v[16], w[16];
        const uint32_t ta = tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)b * WS_ACC_STRIDE +
                            (uint32_t)(c * WS_EPI_CH);
        tmem_ld32(ta, v, w);
        if (c == TNS / WS_EPI_CH - 1) {
          // the accumulator has been read: the next tile's MMAs may overwrite it
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(&accempty[b]);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          wt[lane * WS_EPI_LD + q] = v[q];
          wt[lane * WS_EPI_LD + 16 + q] = w[q];
        }
        __syncwarp();
        // lane = column gj of the chunk, rows Rw + i; every C0 value is loaded before the
        // first store (C may be C0, so the loads could not move past the stores)
        const int gj = c * WS_EPI_CH + lane;
        float c0v[32];
        if (uniform) {
          // the warp's rows are all Re rows or all Im rows of C: one row pointer
          if (gj < p.N) {
            if (C0) {
              const float* q0 = C0 + 2 * ((int64_t)gi0 * p.ldc0 + gj) + comp0;
#pragma unroll
              for (int i = 0; i < 32; ++i) c0v[i] = i < nval ? q0[(int64_t)i * 2 * p.ldc0] : 0.f;
            }
            float* q = C + 2 * ((int64_t)gi0 * p.ldc + gj) + comp0;
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < nval) {
                float res = p.alpha.x * wt[i * WS_EPI_LD + lane];
                if (C0) res = fmaf(p.beta.x, c0v[i], res);
                q[(int64_t)i * 2 * p.ldc] = res;
              }
          }
        } else {
          if (C0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const int R = Rw + i;
              const int gi = R < p.M ? R : R - p.M, comp = R < p.M ? 0 : 1;
              c0v[i] = (R < 2 * p.M && gj < p.N) ? C0[2 * ((int64_t)gi * p.ldc0 + gj) + comp] : 0.f;
            }
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int R = Rw + i;
            const int gi = R < p.M ? R : R - p.M, comp = R < p.M ? 0 : 1;
            if (R < 2 * p.M && gj < p.N) {
              float res = p.alpha.x * wt[i * WS_EPI_LD + lane];
              if (C0) res = fmaf(p.beta.x, c0v[i], res);
              C[2 * ((int64_t)gi * p.ldc + gj) + comp] = res;
            }
          }
        }
        __syncwarp();
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicCAS(p.status, DEV_OK, DEV_TIMEOUT);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(WS_TMEM_COLS)
                 : "memory");
  }
}

int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 1;
    return v > 0 ? v : 1;
  }();
  return n;
}

}  // namespace

static std::atomic<long long> g_wait_limit{WAIT_LIMIT_CYCLES};

long long tc_wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

void tc_set_wait_limit(long long cycles) {
  g_wait_limit.store(cycles > 0 ? cycles : WAIT_LIMIT_CYCLES, std::memory_order_relaxed);
}

cudaError_t launch_tc_cgemm(int M, int N, int K, bool ta, bool tb, float2 alpha, const float2* A,
                            int64_t lda, int64_t sA, const float2* B, int64_t ldb, int64_t sB,
                            float2 beta, const float2* C0, int64_t ldc0, int64_t sC0, float2* C,
                            int64_t ldc, int64_t sC, int batch, int32_t* status, cudaStream_t s,
                            int variant) {
  if (batch <= 0) return cudaSuccess;
  if (batch > 65535 || M < 1 || N < 1 || K < 1) return cudaErrorInvalidValue;
  TcArgs a{M,   N,   K,    A,   lda,   sA,   B,      ldb,   sB, C, ldc, sC, C0,
           ldc0, sC0, alpha, beta, status, batch, tc_wait_limit()};
  dim3 grd((unsigned)ceil_div(N, TNC), (unsigned)ceil_div(M, TM), (unsigned)batch);
  auto launch = [&](auto kern) -> cudaError_t {
    RCI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)SMEM_BYTES));
    kern<<<grd, TC_THREADS, SMEM_BYTES, s>>>(a);
    rci_note_launch();
    return cudaGetLastError();
  };
  if (N <= TNS && alpha.y == 0.f && beta.y == 0.f) {  // real scalars: the stacked form
    if (variant == 0) {
      const cudaError_t e =
          launch_tc_cgemm_tma(M, N, K, ta, tb, alpha.x, A, lda, sA, B, ldb, sB, beta.x, C0, ldc0,
                              sC0, C, ldc, sC, batch, status, tc_wait_limit(), s);
      if (e != cudaErrorNotSupported) return e;
    }
    // persistent: one CTA per SM (or per tile, when there are fewer)
    const int nsm = sm_count();
    const int64_t ntiles = (int64_t)batch * ceil_div(2 * (int64_t)M, TM);
    const unsigned gx = (unsigned)(ntiles < nsm ? ntiles : nsm);
    auto launch_ws = [&](auto kern) -> cudaError_t {
      RCI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)WS_SMEM_BYTES));
      kern<<<gx, WS_THREADS, WS_SMEM_BYTES, s>>>(a);
      rci_note_launch();
      return cudaGetLastError();
    };
    if (!ta && !tb) return launch_ws(tc_cgemm_ws_kernel<false, false>);
    if (!ta && tb) return launch_ws(tc_cgemm_ws_kernel<false, true>);
    if (ta && !tb) return launch_ws(tc_cgemm_ws_kernel<true, false>);
    return launch_ws(tc_cgemm_ws_kernel<true, true>);
  }
  if (!ta && !tb) return launch(tc_cgemm_kernel<false, false>);
  if (!ta && tb) return launch(tc_cgemm_kernel<false, true>);
  if (ta && !tb) return launch(tc_cgemm_kernel<true, false>);
  return launch(tc_cgemm_kernel<true, true>);
}
