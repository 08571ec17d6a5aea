// Tensor-core (tcgen05, 3xTF32) batched complex FP32 GEMM; see tc_gemm.cu.
#pragma once

#include "common.cuh"

// C[z] = alpha op(A[z]) op(B[z]) + beta C0[z] for z < batch (row-major complex64,
// element strides between batch members).  Bounded internal waits: a timeout is
// recorded as DEV_TIMEOUT in *status.
// variant: 0 = the TMA-fed kernel where it applies (real alpha, beta, N <= 160, the
// alignments below), else the register-staged kernels; 1 = register-staged only.
cudaError_t launch_tc_cgemm(int M, int N, int K, bool ta, bool tb, float2 alpha, const float2* A,
                            int64_t lda, int64_t sA, const float2* B, int64_t ldb, int64_t sB,
                            float2 beta, const float2* C0, int64_t ldc0, int64_t sC0, float2* C,
                            int64_t ldc, int64_t sC, int batch, int32_t* status, cudaStream_t s,
                            int variant = 0);

// The TMA-fed form (tc_gemm_tma.cu): real alpha and beta, 2 <= N <= 160 and even, A, B, C,
// C0 16-byte aligned, even leading dimensions and batch strides.  Returns
// cudaErrorNotSupported (nothing launched) where these do not hold.
cudaError_t launch_tc_cgemm_tma(int M, int N, int K, bool ta, bool tb, float alpha,
                                const float2* A, int64_t lda, int64_t sA, const float2* B,
                                int64_t ldb, int64_t sB, float beta, const float2* C0,
                                int64_t ldc0, int64_t sC0, float2* C, int64_t ldc, int64_t sC,
                                int batch, int32_t* status, long long wait_limit, cudaStream_t s);

// One K segment of a TMA-fed product: output z (zlo <= z < zhi) adds op(A[z + zA]) op(B[z + zB])
// over this segment's K, with A and B members 0 .. nA - 1 / nB - 1 at element strides sA, sB.
struct TcSegment {
  const float2* A;
  int64_t lda, sA;
  int nA;
  bool ta;
  const float2* B;
  int64_t ldb, sB;
  int nB;
  bool tb;
  int K;
  int zA, zB, zlo, zhi;
};

// C[z] = alpha sum_g op(A_g[z + zA_g]) op(B_g[z + zB_g]) + beta C0[z] over the segments (one
// or two, each with its own transposes) that include z; same shape and alignment rules as
// launch_tc_cgemm_tma, cudaErrorNotSupported (nothing launched) otherwise.
cudaError_t launch_tc_cgemm_tma_seg(int M, int N, int nseg, const TcSegment* seg, float alpha,
                                    float beta, const float2* C0, int64_t ldc0, int64_t sC0,
                                    float2* C, int64_t ldc, int64_t sC, int batch, int32_t* status,
                                    long long wait_limit, cudaStream_t s);

// One set of products of a TMA-fed launch: C[z] (z < batch) as in launch_tc_cgemm_tma_seg.
struct TcJob {
  int nseg;
  TcSegment seg[2];
  float alpha, beta;
  const float2* C0;
  int64_t ldc0, sC0;
  float2* C;
  int64_t ldc, sC;
  int batch;
};

// One launch over up to two jobs with the same M and N (their tiles numbered job after job);
// a job with batch 0 is skipped.  cudaErrorNotSupported (nothing launched) where any job's
// operands break the TMA rules.
cudaError_t launch_tc_cgemm_tma_jobs(int M, int N, int njob, const TcJob* jobs, int32_t* status,
                                     long long wait_limit, cudaStream_t s);

// Cycles a pipeline wait inside the tensor-core kernels may spin before the kernel gives
// up with DEV_TIMEOUT (process-wide; <= 0 restores the default of 4e9 cycles, ~2 s).  The
// wait for the kernel's own MMAs before its tensor memory is freed always keeps the default.
long long tc_wait_limit();
void tc_set_wait_limit(long long cycles);

// Batched inversion of complex FP32 n x n blocks (n <= 160) with partial pivoting, blocked
// Gauss-Jordan with tensor-core (tcgen05, 3xTF32) panel updates; see tc_gj.cu.  src and out
// are row-major, `stride` complex elements apart; src is not modified.  A zero pivot is
// recorded as DEV_SINGULAR, an expired wait as DEV_TIMEOUT, in *status.  maxabs (or null):
// atomicMax of the bit pattern of the largest |re|, |im| among the blocks' entries.
cudaError_t launch_tc_gj(const float2* src, int64_t src_stride, float2* out, int64_t out_stride,
                         int n, int batch, int32_t* status, cudaStream_t s,
                         uint32_t* maxabs = nullptr);
