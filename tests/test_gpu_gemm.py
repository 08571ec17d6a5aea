"""Batched complex GEMM (the factorisation's products X = Dinv L, Y = Dinv L^T, the Schur
updates D - L Y - L^T X and L' = -L X) through the C ABI: the TMA-fed tensor-core kernel (A
operand in tensor memory), the register-staged tensor-core kernel and the SIMT kernel
against the same product in complex128, at the block sizes of the workloads (128, 160, 224),
ragged sizes below one tile and one K stage, all four transpose combinations, batch strides
that interleave the members (as the factorisation's L + n^2 with stride 2 n^2), more tiles
than SMs, and C0 aliasing C."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2207_10701_gb300 as P  # noqa: E402

RCI_EINVAL = 1


def _rand(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _ref(A, B, C0, alpha, beta, ta, tb):
    a = A.astype(np.complex128)
    b = B.astype(np.complex128)
    if ta:
        a = np.transpose(a, (0, 2, 1))
    if tb:
        b = np.transpose(b, (0, 2, 1))
    out = alpha * (a @ b)
    scale = abs(alpha) * (np.abs(a) @ np.abs(b))
    if C0 is not None:
        out = out + beta * C0.astype(np.complex128)
        scale = scale + abs(beta) * np.abs(C0)
    return out, scale


def _check(got, ref, scale, tol=4e-6):
    # 3xTF32 with FP32 accumulation: the error of each entry is a small multiple of the FP32
    # unit times sum_k |a_ik| |b_kj| (plus |beta c0|)
    err = np.abs(got.astype(np.complex128) - ref)
    bound = tol * (scale + 1e-30)
    worst = float(np.max(err / bound))
    assert worst <= 1.0, worst


def _padded(rng, batch, rows, cols):
    # rows of an even leading dimension (cols rounded up to even), as the TMA boxes need
    full = _rand(rng, (batch, rows, cols + (cols & 1)))
    return full[:, :, :cols], torch.from_numpy(full).cuda()[:, :, :cols]


def _run(M, N, K, batch, ta, tb, alpha, beta, kernel, seed, with_c0=True):
    rng = np.random.default_rng(seed)
    A, tA = _padded(rng, batch, *((K, M) if ta else (M, K)))
    B, tB = _padded(rng, batch, *((N, K) if tb else (K, N)))
    C0, tC0 = _padded(rng, batch, M, N) if with_c0 else (None, None)
    got = P.cgemm_batched(tA, tB, tC0, alpha=alpha, beta=beta, ta=ta, tb=tb,
                          kernel=kernel).cpu().numpy()
    ref, scale = _ref(A, B, C0, alpha, beta, ta, tb)
    _check(got, ref, scale)


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
def test_factor_block_products(kernel, ta, tb):
    # 160 x 160 blocks, more tiles than SMs (3 row tiles x 200 products)
    if kernel == 3 and ta and tb:  # the SIMT kernel has no both-transposed form
        with pytest.raises(P.RciError) as e:
            _run(160, 160, 160, 2, ta, tb, -1.0, 1.0, kernel, seed=0)
        assert e.value.status == RCI_EINVAL
        return
    _run(160, 160, 160, 200, ta, tb, -1.0, 1.0, kernel, seed=1 + 2 * ta + tb)


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("M,N,K", [(128, 128, 128), (224, 160, 224), (100, 98, 37), (1, 2, 1),
                                   (65, 16, 9), (64, 160, 8), (160, 158, 161), (33, 30, 200)])
def test_ragged_and_workload_sizes(kernel, M, N, K):
    # (small batches: kernel 0 dispatches these to SIMT, which has no both-transposed form)
    combos = [(False, False), (True, False), (False, True)] + ([(True, True)] if kernel else [])
    for ta, tb in combos:
        _run(M, N, K, 3, ta, tb, 0.5, -2.0, kernel, seed=M * 7 + N * 3 + K)


@pytest.mark.parametrize("kernel", [0, 2])
def test_without_c0_and_interleaved_batch_strides(kernel):
    # A and B are every other block of one array (element stride 2 n^2 between members), as
    # the factorisation passes L + n^2; no C0
    n, batch = 160, 160
    rng = np.random.default_rng(5)
    big_a = _rand(rng, (2 * batch, n, n))
    big_b = _rand(rng, (2 * batch, n, n))
    ta_ = torch.from_numpy(big_a).cuda()[1::2]
    tb_ = torch.from_numpy(big_b).cuda()[0::2]
    assert ta_.stride(0) == 2 * n * n
    got = P.cgemm_batched(ta_, tb_, None, alpha=-1.0, kernel=kernel).cpu().numpy()
    ref, scale = _ref(big_a[1::2], big_b[0::2], None, -1.0, 0.0, False, False)
    _check(got, ref, scale)


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_c0_aliasing_c(kernel):
    # D' -= L^T X computed in place (C0 is C), as the second Schur update does
    n, batch = 160, 50
    rng = np.random.default_rng(9)
    A, B, D = _rand(rng, (batch, n, n)), _rand(rng, (batch, n, n)), _rand(rng, (batch, n, n))
    td = torch.from_numpy(D).cuda()
    P.cgemm_batched(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), td, alpha=-1.0,
                    beta=1.0, ta=True, kernel=kernel, out=td)
    ref, scale = _ref(A, B, D, -1.0, 1.0, True, False)
    _check(td.cpu().numpy(), ref, scale)


def test_tma_kernel_rejects_what_it_cannot_take():
    rng = np.random.default_rng(3)
    for N in (7, 162):  # odd N, N above one accumulator
        A = torch.from_numpy(_rand(rng, (2, 16, 16))).cuda()
        B = torch.from_numpy(_rand(rng, (2, 16, N))).cuda()
        with pytest.raises(P.RciError) as e:
            P.cgemm_batched(A, B, kernel=2)
        assert e.value.status == RCI_EINVAL
        # the other kernels take it
        got = P.cgemm_batched(A, B, kernel=0).cpu().numpy()
        ref, scale = _ref(A.cpu().numpy(), B.cpu().numpy(), None, 1.0, 0.0, False, False)
        _check(got, ref, scale)


def test_fp64_products_simt():
    rng = np.random.default_rng(4)
    A = (rng.standard_normal((4, 96, 80)) + 1j * rng.standard_normal((4, 96, 80)))
    B = (rng.standard_normal((4, 80, 72)) + 1j * rng.standard_normal((4, 80, 72)))
    got = P.cgemm_batched(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), kernel=0)
    ref = A @ B
    assert np.max(np.abs(got.cpu().numpy() - ref)) < 1e-12 * np.max(np.abs(A) @ np.abs(B))
