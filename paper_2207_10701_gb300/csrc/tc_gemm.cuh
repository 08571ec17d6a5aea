// Tensor-core (tcgen05, 3xTF32) batched complex FP32 GEMM; see tc_gemm.cu.
#pragma once

#include "common.cuh"

// C[z] = alpha op(A[z]) op(B[z]) + beta C0[z] for z < batch (row-major complex64,
// element strides between batch members).  Bounded internal waits: a timeout is
// recorded as DEV_TIMEOUT in *status.
cudaError_t launch_tc_cgemm(int M, int N, int K, bool ta, bool tb, float2 alpha, const float2* A,
                            int64_t lda, int64_t sA, const float2* B, int64_t ldb, int64_t sB,
                            float2 beta, const float2* C0, int64_t ldc0, int64_t sC0, float2* C,
                            int64_t ldc, int64_t sC, int batch, int32_t* status, cudaStream_t s);

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
