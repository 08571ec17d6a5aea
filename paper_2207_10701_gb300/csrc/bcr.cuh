// Block cyclic reduction (BCR) direct solver for the block-tridiagonal FDFD operator.
//
// A (ordered x-outermost) has nx block rows i with a tridiagonal ny x ny diagonal
// block T_i and diagonal couplings diag(cx[i-1]) (to i-1) and diag(cx[i]) (to i+1).
// A = A^T, so every reduced system stays symmetric and only the lower coupling L_i
// (block (i, i-1)) is kept; the upper one is L_{i+1}^T.
//
// One reduction level eliminates the odd rows r of the current system:
//   X_r = D_r^{-1} L_r,  Y_r = D_r^{-1} L_{r+1}^T
//   kept row e:  D'_e = D_e - L_e Y_{e-1} - L_{e+1}^T X_{e+1},   L'_e = -L_e X_{e-1}
// Solve, forward:  t_r = D_r^{-1} b_r,   b'_e = b_e - Y_{e-1}^T b_{e-1} - X_{e+1}^T b_{e+1}
//        backward: x_r = t_r - X_r x_{r-1} - Y_r x_{r+1}.
// Level 0 works on the tridiagonal T_i directly (pivoted tridiagonal LU, O(ny^2) per
// row to form the dense Schur blocks); levels >= 1 use explicit inverses from a
// pivoted Gauss-Jordan inversion and batched complex GEMMs.
#pragma once

#include <vector>

#include "common.cuh"

struct BcrHandle;

// prec: RCI_FP64 -> double, RCI_FP32_REFINE -> float.  Allocates the factor store from
// mem (cudaMalloc when mem is null).  No kernel is launched.
cudaError_t bcr_create(int nx, int ny, int prec, const DevMem* mem, BcrHandle** out, size_t* bytes);
// Allocate the solve workspace for nrhs right-hand sides now (otherwise the first solve
// with more right-hand sides than before allocates it).
cudaError_t bcr_reserve_ws(BcrHandle* h, int nrhs);
void bcr_destroy(BcrHandle* h);
size_t bcr_bytes(const BcrHandle* h);

// Factor from the FP64 coefficient arrays (dg, cx, cy as in assemble.cu).
cudaError_t bcr_factor(BcrHandle* h, const double2* dg, const double2* cx, const double2* cy,
                       cudaStream_t s);
// Solve A x = b for nrhs right-hand sides, [i][j][q] with leading dimension nrhs, in the
// handle's precision (float2 or double2 buffers).  b and x must not overlap.
cudaError_t bcr_solve(BcrHandle* h, const double2* cx, const void* b, void* x, int nrhs,
                      cudaStream_t s);
// Device status word (DEV_OK / DEV_SINGULAR / DEV_NONFINITE), read synchronously; with
// growth, also the growth estimate of the last factorisation: the largest |re|, |im| of the
// blocks it inverted (the Schur complements of every level) over that of A's coefficients.
cudaError_t bcr_read_status(BcrHandle* h, int32_t* st, cudaStream_t s, double* growth = nullptr);
int bcr_precision(const BcrHandle* h);
// Arithmetic of an FP32 handle from its next bcr_factor on: false (the default) runs the block
// inversions and the products of the factorisation and of the several-right-hand-side solve
// on the tensor cores (3xTF32 products accumulated in FP32, about 3.5 times the error of one
// FP32 rounding per product); true runs them on the FP32 SIMT pipe (the Gauss-Jordan and
// GEMM kernels of this file: one rounding per FMA, several times slower).  FP64 handles
// ignore it.
void bcr_set_simt(BcrHandle* h, bool simt);
bool bcr_simt(const BcrHandle* h);
// Optional profiler (owned by the caller) for the factor / solve kernel families.
void bcr_set_profiler(BcrHandle* h, Profiler* p);

// Batched inverse of complex n x n blocks (row-major, contiguous): prec as the handle's;
// kernel 0 = the factorisation's choice, 1 = SIMT Gauss-Jordan, 2 = tensor-core Gauss-Jordan
// (FP32, n <= 160).  A zero pivot is recorded in *status (device word).
cudaError_t bcr_block_inverse(const void* src, void* out, int n, int batch, int prec, int kernel,
                              int32_t* status, cudaStream_t s);

// Batched complex GEMM C[z] = alpha op(A[z]) op(B[z]) + beta C0[z] (real alpha, beta; prec as
// the handle's; C0 may be null): kernel 0 = the factorisation's dispatch, 1 = tensor cores
// with register-staged operands, 2 = tensor cores fed by TMA with A in tensor memory,
// 3 = SIMT.  An expired wait is recorded as DEV_TIMEOUT in *status (device word).
cudaError_t bcr_gemm(int M, int N, int K, bool ta, bool tb, double alpha, const void* A,
                     int64_t lda, int64_t sA, const void* B, int64_t ldb, int64_t sB, double beta,
                     const void* C0, int64_t ldc0, int64_t sC0, void* C, int64_t ldc, int64_t sC,
                     int batch, int prec, int kernel, int32_t* status, cudaStream_t s);
