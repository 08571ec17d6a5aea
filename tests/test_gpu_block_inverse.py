"""Batched block inversion (the factorisation's block-inverse step) through the C ABI:
the tensor-core Gauss-Jordan kernel and the SIMT one against numpy's inverse (LAPACK) of
the same blocks in complex128, at sizes that span one panel, ragged panels, the two- and
three-tile tensor-memory layouts and a batch larger than the SM count; exact cases
(identity, permutation) and a singular block."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2207_10701_gb300 as P  # noqa: E402


def _blocks(n, batch, seed, shift=2.0):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    a += shift * np.sqrt(n) * np.exp(1j * rng.uniform(0, 2 * np.pi, (batch, 1, 1))) * np.eye(n)
    return a


def _rel_err(x, ref):
    return float(np.max(np.linalg.norm(x - ref, axis=(1, 2)) / np.linalg.norm(ref, axis=(1, 2))))


@pytest.mark.parametrize("n", [1, 7, 16, 33, 100, 128, 129, 144, 160])
@pytest.mark.parametrize("kernel", [1, 2])
def test_fp32_block_inverse_matches_lapack(n, kernel):
    a = _blocks(n, 6, n)
    a32 = a.astype(np.complex64)
    ref = np.linalg.inv(a32.astype(np.complex128))
    got = P.block_inverse(torch.from_numpy(a32).cuda(), kernel=kernel).cpu().numpy()
    assert _rel_err(got, ref) < 2e-5, _rel_err(got, ref)


def test_tensor_core_and_simt_kernels_agree_on_a_large_batch():
    # more blocks than SMs: the persistent tensor-core kernel loops over its share
    a = _blocks(160, 400, 11, shift=1.0).astype(np.complex64)
    t = torch.from_numpy(a).cuda()
    tc = P.block_inverse(t, kernel=2).cpu().numpy()
    simt = P.block_inverse(t, kernel=1).cpu().numpy()
    ref = np.linalg.inv(a.astype(np.complex128))
    # these blocks are less well conditioned: both FP32 kernels lose digits alike, and the
    # tensor-core one (3xTF32 updates) must stay within a small factor of the SIMT one
    e_tc, e_simt = _rel_err(tc, ref), _rel_err(simt, ref)
    assert e_tc < max(3.0 * e_simt, 2e-5), (e_tc, e_simt)


@pytest.mark.parametrize("n", [16, 128, 160])
def test_exact_cases(n):
    rng = np.random.default_rng(n)
    perm = rng.permutation(n)
    Pm = np.eye(n)[perm] * (1 + 1j)               # scaled permutation: inverse exact in FP32
    eye = np.eye(n)
    a = np.stack([eye, Pm]).astype(np.complex64)
    got = P.block_inverse(torch.from_numpy(a).cuda(), kernel=2).cpu().numpy()
    assert np.array_equal(got[0], eye.astype(np.complex64))
    assert np.array_equal(got[1], np.linalg.inv(Pm).astype(np.complex64))


def test_singular_block_is_reported():
    a = _blocks(48, 3, 5).astype(np.complex64)
    a[1] = 0
    with pytest.raises(P.RciError) as ei:
        P.block_inverse(torch.from_numpy(a).cuda(), kernel=2)
    assert ei.value.status == 5                    # RCI_ESINGULAR
