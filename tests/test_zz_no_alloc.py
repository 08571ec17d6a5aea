"""The allocation-free quadratic-form entry point (rci_qform_toeplitz_noalloc).

It exists for callers that must not allocate device memory: code that hands all of HBM
to its own pool, or that keeps several streams busy and cannot afford the device-wide
synchronisation of cudaFree.  Its scratch is a fixed array inside the library, shared by
all calls.  These tests call it through the C ABI and check it against the allocating
entry point rci_qform_toeplitz at the quadratic-form tolerance (1e-12 relative), on two
calls in a row with different sizes (the second must not see the first call's scratch).
The file is named so that pytest collects it last."""
import ctypes as C
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2207_10701_gb300 as P  # noqa: E402
from paper_2207_10701_gb300 import build as B  # noqa: E402

TOL = 1e-12


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    k_s, h = 2 * math.pi * math.sqrt(2.1), 0.05
    m = np.arange(n)
    lags = np.sinc(k_s * h * m * math.sin(0.35) / math.pi) * math.sin(0.35) / 0.35
    return (torch.from_numpy(v).to("cuda").contiguous(),
            torch.from_numpy(lags).to("cuda").contiguous())


def _ptr(t):
    return C.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.lib()


def test_noalloc_matches_allocating_entry_point_on_two_calls(lib):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, seed in ((20000, 1), (777, 2)):          # large first, then small
        v, lags = _inputs(n, seed)
        ref = P.qform_toeplitz(v, lags)              # existing (allocating) entry point
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.rci_qform_toeplitz_noalloc(_ptr(v), _ptr(lags), n, _ptr(out), stream)
        assert st == 0, P.rci.STATUS.get(st)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= TOL * abs(ref), (n, got, ref)


def test_noalloc_call_leaves_device_memory_unchanged(lib):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    v, lags = _inputs(4000, 3)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    assert lib.rci_qform_toeplitz_noalloc(_ptr(v), _ptr(lags), 4000, _ptr(out), stream) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert lib.rci_qform_toeplitz_noalloc(_ptr(v), _ptr(lags), 4000, _ptr(out), stream) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert abs(float(out.item()) - P.qform_toeplitz(v, lags)) <= TOL * abs(float(out.item()))


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    n = P.QFORM_NOALLOC_MAX_N + 1
    v, lags = _inputs(n, 4)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    st = lib.rci_qform_toeplitz_noalloc(_ptr(v), _ptr(lags), n, _ptr(out), None)
    assert st == 1                                   # RCI_EINVAL
    assert float(out.item()) == -1.0
    with pytest.raises(P.RciError):
        P.qform_toeplitz_noalloc(v, lags, out)


@pytest.mark.parametrize("n", [P.QFORM_NOALLOC_MAX_N, 1, 100])
def test_noalloc_at_the_size_limits_of_its_scratch(lib, n):
    # n = the maximum fills the scratch array to its last partial; n < 128 is a single,
    # partial tile
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    v, lags = _inputs(n, 10 + n % 7)
    ref = P.qform_toeplitz(v, lags)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    assert lib.rci_qform_toeplitz_noalloc(_ptr(v), _ptr(lags), n, _ptr(out), stream) == 0
    torch.cuda.synchronize()
    got = float(out.item())
    assert abs(got - ref) <= TOL * abs(ref), (n, got, ref)


def test_noalloc_binding_rejects_tensors_the_kernel_cannot_address(lib):
    v, lags = _inputs(64, 5)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        P.qform_toeplitz_noalloc(v, lags, torch.empty(1, dtype=torch.float64))   # host out
    with pytest.raises(ValueError):
        P.qform_toeplitz_noalloc(v.cpu(), lags, out)                             # host v
    with pytest.raises(ValueError):
        P.qform_toeplitz_noalloc(v, lags[:10].contiguous(), out)                 # short lags
    with pytest.raises(ValueError):
        P.qform_toeplitz_noalloc(v, lags, torch.empty(0, dtype=torch.float64, device="cuda"))
    P.qform_toeplitz_noalloc(v, lags, out)
    torch.cuda.synchronize()
    ref = P.qform_toeplitz(v, lags)
    assert abs(float(out.item()) - ref) <= TOL * abs(ref)
