"""ctypes binding of include/rci.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librci.so")

OBJ_POINT, OBJ_PLANEWAVE, OBJ_VIRTUAL_FOCUS, OBJ_USER_ROW = 0, 1, 2, 3
LIGHT_CONE, LIGHT_ANNULUS, LIGHT_USER_LAGS, LIGHT_TABULATED = 0, 1, 2, 3
FP64, FP32_REFINE = 0, 1

STATUS = {0: "RCI_OK", 1: "RCI_EINVAL", 2: "RCI_ENOMEM", 3: "RCI_ECUDA", 4: "RCI_ESTATE",
          5: "RCI_ESINGULAR", 6: "RCI_ENOCONV", 7: "RCI_ENUMERIC", 8: "RCI_ETIMEOUT"}


class GridDescC(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("ny", C.c_int32), ("ppl", C.c_int32),
                ("cell_px", C.c_int32), ("npml", C.c_int32), ("rows_sub", C.c_int32),
                ("rows_pillar", C.c_int32), ("src_offset", C.c_int32),
                ("eps_pillar", C.c_double), ("eps_sub", C.c_double), ("eps_air", C.c_double),
                ("pml_R0", C.c_double), ("pml_m", C.c_int32), ("prec", C.c_int32),
                ("device", C.c_int32), ("reserved", C.c_int32)]


class ObjectiveC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("monitor_row", C.c_int32), ("i_f", C.c_int32),
                ("j_f", C.c_int32), ("theta_out", C.c_double), ("x_f", C.c_double),
                ("d_rows", C.c_int32), ("reserved", C.c_int32),
                ("w_row", C.POINTER(C.c_double))]


class LightC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("c", C.c_double),
                ("th1", C.c_double), ("th2", C.c_double), ("lags", C.POINTER(C.c_double)),
                ("tab_theta", C.POINTER(C.c_double)), ("tab_rho", C.POINTER(C.c_double)),
                ("n_tab", C.c_int64)]


class InfoC(C.Structure):
    _fields_ = [("refine_iters", C.c_int32), ("fallback", C.c_int32),
                ("rel_residual", C.c_double), ("ms_factor", C.c_double),
                ("ms_solve", C.c_double), ("ms_qform", C.c_double),
                ("growth_est", C.c_double), ("krylov_steps", C.c_int32),
                ("simt_refactor", C.c_int32)]


class ServerDescC(C.Structure):
    _fields_ = [("device", C.c_int32), ("slots", C.c_int32), ("arena_bytes", C.c_uint64),
                ("cache_bytes", C.c_uint64), ("lookahead", C.c_int32), ("reserved", C.c_int32)]


class RequestC(C.Structure):
    _fields_ = [("grid", GridDescC), ("widths", C.POINTER(C.c_double)), ("obj", ObjectiveC),
                ("light", LightC), ("want_grad", C.c_int32), ("reserved", C.c_int32),
                ("design_key", C.c_uint64), ("grad_out", C.POINTER(C.c_double))]


class ResultC(C.Structure):
    _fields_ = [("status", C.c_int32), ("cache_hit", C.c_int32), ("value", C.c_double),
                ("refine_iters", C.c_int32), ("fp64_fallback", C.c_int32),
                ("rel_residual", C.c_double), ("t_submit_us", C.c_double),
                ("t_start_us", C.c_double), ("t_end_us", C.c_double),
                ("footprint", C.c_uint64), ("simt_refactor", C.c_int32),
                ("reserved", C.c_int32)]


class ServerStatsC(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "failed", "cache_hits",
                                          "cache_evictions", "admission_waits", "bypasses")] + \
               [(n, C.c_int32) for n in ("in_flight", "queued", "resident", "reserved")] + \
               [(n, C.c_uint64) for n in ("arena_bytes", "arena_used", "arena_peak",
                                          "cache_bytes")]


PROFILE_FAMILIES = ["level0", "invert", "gemm", "solve", "residual", "qform", "setup", "grad"]


class ProfileC(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("flops", C.c_double * 8), ("bytes", C.c_double * 8),
                ("launches", C.c_int64 * 8)]


class PeaksC(C.Structure):
    _fields_ = [("fp32_fma_tflops", C.c_double), ("fp64_fma_tflops", C.c_double),
                ("fp64_dmma_tflops", C.c_double), ("int8_imma_tops", C.c_double),
                ("tf32_tcgen05_tflops", C.c_double), ("bf16_tcgen05_tflops", C.c_double),
                ("sm_count", C.c_int32), ("reserved", C.c_int32)]


@dataclasses.dataclass
class Info:
    refine_iters: int
    rel_residual: float
    ms_factor: float
    ms_solve: float
    ms_qform: float
    fallback: bool = False
    growth_est: float = 0.0
    krylov_steps: int = 0
    simt_refactor: bool = False

    @staticmethod
    def of(c: InfoC) -> "Info":
        return Info(c.refine_iters, c.rel_residual, c.ms_factor, c.ms_solve, c.ms_qform,
                    bool(c.fallback), c.growth_est, c.krylov_steps, bool(c.simt_refactor))


class RciError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_P = C.c_void_p
_D = C.POINTER(C.c_double)
EXPORTED = {
    "rci_create_grid": (C.c_int, [C.POINTER(GridDescC), _P, C.POINTER(_P)]),
    "rci_destroy_grid": (C.c_int, [_P]),
    "rci_grid_query": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64), C.POINTER(C.c_size_t)]),
    "rci_set_design": (C.c_int, [_P, _P, C.c_int64, C.c_int]),
    "rci_factor": (C.c_int, [_P]),
    "rci_set_refinement": (C.c_int, [_P, C.c_double, C.c_int32]),
    "rci_solve": (C.c_int, [_P, _P, _P, C.c_int64, C.POINTER(InfoC)]),
    "rci_solve_reciprocal": (C.c_int, [_P, C.POINTER(ObjectiveC), _P, _P, C.POINTER(InfoC)]),
    "rci_avg_intensity": (C.c_int, [_P, C.POINTER(ObjectiveC), C.POINTER(LightC), _D,
                                    C.POINTER(InfoC)]),
    "rci_avg_intensity_grad": (C.c_int, [_P, C.POINTER(ObjectiveC), C.POINTER(LightC), _D, _D,
                                         C.POINTER(InfoC)]),
    "rci_avg_intensity_correlated": (C.c_int, [_P, C.POINTER(ObjectiveC), _D, _D, C.c_int64, _D,
                                               _D, C.POINTER(InfoC)]),
    "rci_avg_intensity_dense": (C.c_int, [_P, C.POINTER(ObjectiveC), _P, _D, C.POINTER(InfoC)]),
    "rci_avg_intensity_multi": (C.c_int, [_P, C.POINTER(ObjectiveC), C.c_int64, C.POINTER(LightC),
                                          _D, _D, C.POINTER(InfoC)]),
    "rci_solve_angles": (C.c_int, [_P, C.POINTER(ObjectiveC), _D, _D, C.c_int64, _D, _D,
                                   C.POINTER(InfoC)]),
    "rci_avg_bruteforce": (C.c_int, [_P, C.POINTER(ObjectiveC), C.POINTER(LightC), C.c_int64,
                                     _D, _D, C.POINTER(InfoC)]),
    "rci_qform_toeplitz": (C.c_int, [_P, _P, C.c_int64, _D, _P]),
    "rci_qform_toeplitz_noalloc": (C.c_int, [_P, _P, C.c_int64, _P, _P]),
    "rci_gauss_legendre": (C.c_int, [C.c_int64, C.c_double, C.c_double, _P, _P, _P]),
    "rci_get_eps": (C.c_int, [_P, _P]),
    "rci_apply_operator": (C.c_int, [_P, _P, _P]),
    "rci_grid_footprint": (C.c_int, [C.POINTER(GridDescC), C.c_int, C.POINTER(C.c_size_t)]),
    "rci_server_create": (C.c_int, [C.POINTER(ServerDescC), C.POINTER(_P)]),
    "rci_server_submit": (C.c_int, [_P, C.POINTER(RequestC), C.POINTER(C.c_uint64)]),
    "rci_server_wait": (C.c_int, [_P, C.c_uint64, C.c_double, C.POINTER(ResultC)]),
    "rci_server_stats_read": (C.c_int, [_P, C.POINTER(ServerStatsC)]),
    "rci_server_destroy": (C.c_int, [_P]),
    "rci_profile_enable": (C.c_int, [_P, C.c_int]),
    "rci_profile_read": (C.c_int, [_P, C.POINTER(ProfileC)]),
    "rci_kernel_launches": (C.c_uint64, []),
    "rci_set_wait_limit": (C.c_int64, [C.c_int64]),
    "rci_block_inverse": (C.c_int, [_P, _P, C.c_int64, C.c_int64, C.c_int32, C.c_int32, _P]),
    "rci_cgemm_batched": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_int32,
                                    C.c_double, _P, C.c_int64, C.c_int64, _P, C.c_int64,
                                    C.c_int64, C.c_double, _P, C.c_int64, C.c_int64, _P,
                                    C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_int32, _P]),
    "rci_measure_peaks": (C.c_int, [C.c_int, C.POINTER(PeaksC)]),
    "rci_status_str": (C.c_char_p, [C.c_int]),
    "rci_last_error": (C.c_char_p, [_P]),
}

_lib = None


def lib(path: str = LIB_PATH):
    """Load librci.so (once).  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing; build it with "
                               "`python -m paper_2207_10701_gb300.build`")
        L = C.CDLL(path)
        for name, (res, args) in EXPORTED.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _check(st: int, handle=None):
    if st != 0:
        msg = lib().rci_last_error(handle).decode() if handle else ""
        if not msg:
            msg = lib().rci_status_str(st).decode()
        raise RciError(st, msg)


def _dptr(t):
    return C.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _desc(d, prec=None, device=0) -> GridDescC:
    return GridDescC(d.n_cells, d.ny, d.ppl, d.cell_px, d.npml, d.rows_sub, d.rows_pillar,
                     d.src_offset, d.eps_pillar, d.eps_sub, d.eps_air, d.pml_R0, d.pml_m,
                     d.prec if prec is None else prec, device, 0)


def _objective(o, keep):
    w = None
    if getattr(o, "kind", None) == OBJ_USER_ROW:
        w = np.ascontiguousarray(np.asarray(o.w_row, dtype=np.complex128)).view(np.float64)
        keep.append(w)
    return ObjectiveC(o.kind, o.monitor_row, o.i_f, o.j_f, o.theta_out, o.x_f, o.d_rows, 0,
                      _hptr(w) if w is not None else None)


def _light(L, keep):
    lags = th = rh = None
    if L.kind == LIGHT_USER_LAGS:
        lags = np.ascontiguousarray(np.asarray(L.lags, dtype=np.float64))
        keep.append(lags)
    if L.kind == LIGHT_TABULATED:
        th = np.ascontiguousarray(np.asarray(L.theta, dtype=np.float64))
        rh = np.ascontiguousarray(np.asarray(L.rho, dtype=np.float64))
        if th.shape != rh.shape or th.ndim != 1:
            raise ValueError("tabulated light: theta and rho of equal length")
        keep.extend((th, rh))
    return LightC(L.kind, 0, L.c, L.th1, L.th2, _hptr(lags) if lags is not None else None,
                  _hptr(th) if th is not None else None, _hptr(rh) if rh is not None else None,
                  th.size if th is not None else 0)


class Grid:
    """One geometry on one CUDA device (owns the operator, the factorisation and the
    work buffers).  ``desc`` is any object with the fields of rci_grid_desc."""

    def __init__(self, desc, prec=None, device: int = 0, stream=None):
        torch = _torch()
        self.device = device
        self.torch_device = torch.device("cuda", device)
        self._stream = _stream(stream)
        h = C.c_void_p()
        _check(lib().rci_create_grid(C.byref(_desc(desc, prec, device)), self._stream, C.byref(h)))
        self._h = h
        nx, ny, ns, by = C.c_int64(), C.c_int64(), C.c_int64(), C.c_size_t()
        _check(lib().rci_grid_query(h, C.byref(nx), C.byref(ny), C.byref(ns), C.byref(by)), h)
        self.nx, self.ny, self.n_src = nx.value, ny.value, ns.value
        self.N = self.nx * self.ny
        self.n_cells = int(desc.n_cells)

    def close(self):
        if getattr(self, "_h", None):
            lib().rci_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def profile(self, on: bool = True):
        """Start (reset) or stop bracketing kernel families with CUDA events."""
        _check(lib().rci_profile_enable(self._h, 1 if on else 0), self._h)

    def profile_read(self) -> dict:
        """{family: {"ms", "flops", "bytes", "launches"}} accumulated since profile(True)."""
        p = ProfileC()
        _check(lib().rci_profile_read(self._h, C.byref(p)), self._h)
        return {f: {"ms": p.ms[i], "flops": p.flops[i], "bytes": p.bytes[i],
                    "launches": p.launches[i]} for i, f in enumerate(PROFILE_FAMILIES)}

    def device_bytes(self) -> int:
        by = C.c_size_t()
        _check(lib().rci_grid_query(self._h, None, None, None, C.byref(by)), self._h)
        return by.value

    def set_design(self, widths):
        torch = _torch()
        if isinstance(widths, torch.Tensor) and widths.is_cuda:
            w = widths.to(torch.float64).contiguous()
            _check(lib().rci_set_design(self._h, _dptr(w), w.numel(), 1), self._h)
        else:
            w = np.ascontiguousarray(np.asarray(widths, dtype=np.float64))
            _check(lib().rci_set_design(self._h, w.ctypes.data_as(_P), w.size, 0), self._h)

    def factor(self):
        _check(lib().rci_factor(self._h), self._h)

    def set_refinement(self, tol: float, max_steps: int):
        _check(lib().rci_set_refinement(self._h, tol, max_steps), self._h)

    def solve(self, b, nrhs: int = 1):
        """b: complex128 CUDA tensor of nx*ny*nrhs entries ([i][j][q]); returns x."""
        torch = _torch()
        b = b.to(torch.complex128).contiguous()
        x = torch.empty_like(b)
        info = InfoC()
        _check(lib().rci_solve(self._h, _dptr(b), _dptr(x), nrhs, C.byref(info)), self._h)
        return x, Info.of(info)

    def solve_reciprocal(self, obj, full: bool = False):
        torch = _torch()
        keep = []
        oc = _objective(obj, keep)
        v = torch.empty(self.n_src, dtype=torch.complex128, device=self.torch_device)
        vf = torch.empty(self.N, dtype=torch.complex128, device=self.torch_device) if full else None
        info = InfoC()
        _check(lib().rci_solve_reciprocal(self._h, C.byref(oc), _dptr(v),
                                          _dptr(vf) if full else None, C.byref(info)), self._h)
        return (v, vf, Info.of(info)) if full else (v, Info.of(info))

    def avg_intensity(self, obj, light):
        keep = []
        oc, lc = _objective(obj, keep), _light(light, keep)
        out = C.c_double()
        info = InfoC()
        _check(lib().rci_avg_intensity(self._h, C.byref(oc), C.byref(lc), C.byref(out),
                                       C.byref(info)), self._h)
        return out.value, Info.of(info)

    def avg_intensity_grad(self, obj, light):
        """(F, dF/d widths as float64[n_cells], Info): the adjoint gradient of Eq. 7
        (one extra refined solve on the same factorisation)."""
        keep = []
        oc, lc = _objective(obj, keep), _light(light, keep)
        out = C.c_double()
        grad = np.empty(self.n_cells)
        info = InfoC()
        _check(lib().rci_avg_intensity_grad(self._h, C.byref(oc), C.byref(lc), C.byref(out),
                                            _hptr(grad), C.byref(info)), self._h)
        return out.value, grad, Info.of(info)

    def avg_intensity_correlated(self, obj, theta, weight, corr):
        """F for correlated light: corr[q][q'] = <a(theta_q) a*(theta_q')> on the rule
        (theta, weight)."""
        keep = []
        oc = _objective(obj, keep)
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        wq = np.ascontiguousarray(np.asarray(weight, dtype=np.float64))
        cm = np.ascontiguousarray(np.asarray(corr, dtype=np.complex128)).view(np.float64)
        if cm.size != 2 * th.size * th.size or wq.size != th.size:
            raise ValueError("corr must be nq x nq and weight nq long")
        out = C.c_double()
        info = InfoC()
        _check(lib().rci_avg_intensity_correlated(self._h, C.byref(oc), _hptr(th), _hptr(wq),
                                                  th.size, _hptr(cm), C.byref(out),
                                                  C.byref(info)), self._h)
        return out.value, Info.of(info)

    def avg_intensity_dense(self, obj, W):
        """F = v^dag W v for a dense Hermitian W (complex128 CUDA tensor, n_src x n_src)."""
        torch = _torch()
        keep = []
        oc = _objective(obj, keep)
        Wt = W.to(torch.complex128).contiguous()
        if Wt.numel() != self.n_src * self.n_src or not Wt.is_cuda:
            raise ValueError("W must be a CUDA tensor of n_src x n_src entries")
        out = C.c_double()
        info = InfoC()
        _check(lib().rci_avg_intensity_dense(self._h, C.byref(oc), _dptr(Wt), C.byref(out),
                                             C.byref(info)), self._h)
        return out.value, Info.of(info)

    def avg_intensity_multi(self, objectives, light):
        """(F per objective, their sum, Info): one multi-RHS reciprocal solve."""
        keep = []
        arr = (ObjectiveC * len(objectives))(*[_objective(o, keep) for o in objectives])
        lc = _light(light, keep)
        F = np.empty(len(objectives))
        tot = C.c_double()
        info = InfoC()
        _check(lib().rci_avg_intensity_multi(self._h, arr, len(objectives), C.byref(lc), _hptr(F),
                                             C.byref(tot), C.byref(info)), self._h)
        return F, tot.value, Info.of(info)

    def solve_angles(self, obj, theta, weight):
        keep = []
        oc = _objective(obj, keep)
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        wq = np.ascontiguousarray(np.asarray(weight, dtype=np.float64))
        f = np.empty(th.size)
        avg = C.c_double()
        info = InfoC()
        _check(lib().rci_solve_angles(self._h, C.byref(oc), _hptr(th), _hptr(wq), th.size,
                                      _hptr(f), C.byref(avg), C.byref(info)), self._h)
        return avg.value, f, Info.of(info)

    def avg_bruteforce(self, obj, light, nq: int):
        keep = []
        oc, lc = _objective(obj, keep), _light(light, keep)
        f = np.empty(nq)
        avg = C.c_double()
        info = InfoC()
        _check(lib().rci_avg_bruteforce(self._h, C.byref(oc), C.byref(lc), nq, _hptr(f),
                                        C.byref(avg), C.byref(info)), self._h)
        return avg.value, f, Info.of(info)

    def eps(self):
        torch = _torch()
        e = torch.empty(self.N, dtype=torch.float64, device=self.torch_device)
        _check(lib().rci_get_eps(self._h, _dptr(e)), self._h)
        return e.view(self.nx, self.ny)

    def apply_operator(self, x):
        torch = _torch()
        x = x.to(torch.complex128).contiguous()
        y = torch.empty_like(x)
        _check(lib().rci_apply_operator(self._h, _dptr(x), _dptr(y)), self._h)
        return y


def kernel_launches() -> int:
    """Kernels launched by librci in this process so far."""
    return int(lib().rci_kernel_launches())


def measure_peaks(device: int = 0) -> dict:
    """Measured arithmetic peaks of the device (rci_measure_peaks), rates in 1e12 ops/s."""
    p = PeaksC()
    _check(lib().rci_measure_peaks(device, C.byref(p)))
    return {n: getattr(p, n) for n, _ in PeaksC._fields_ if n != "reserved"}


def block_inverse(blocks, kernel: int = 0, stream=None):
    """Inverses of a batch of complex blocks (CUDA tensor [batch, n, n], complex64 or
    complex128) with the factorisation's block-inverse kernels (rci_block_inverse);
    kernel 0 = its choice, 1 = SIMT, 2 = tensor cores (complex64, n <= 160)."""
    torch = _torch()
    if blocks.dim() != 3 or blocks.shape[1] != blocks.shape[2] or not blocks.is_cuda:
        raise ValueError("blocks: CUDA tensor [batch, n, n]")
    if blocks.dtype not in (torch.complex64, torch.complex128):
        raise TypeError("complex64 or complex128 blocks")
    src = blocks.contiguous().clone()
    out = torch.empty_like(src)
    prec = FP32_REFINE if src.dtype == torch.complex64 else FP64
    _check(lib().rci_block_inverse(_dptr(src), _dptr(out), src.shape[1], src.shape[0], prec,
                                   kernel, _stream(stream)))
    return out


def cgemm_batched(A, B, C0=None, alpha: float = 1.0, beta: float = 0.0, ta: bool = False,
                  tb: bool = False, kernel: int = 0, out=None, stream=None):
    """C[z] = alpha op(A[z]) op(B[z]) + beta C0[z] with the factorisation's batched complex
    GEMM kernels (rci_cgemm_batched): CUDA tensors [batch, rows, cols] of complex64 or
    complex128 whose rows are contiguous (any row and batch strides); op = transpose when ta
    / tb.  kernel 0 = the factorisation's dispatch, 1 = tensor cores with register-staged
    operands, 2 = tensor cores fed by TMA, 3 = SIMT.  Returns C (`out` when given)."""
    torch = _torch()
    for t in (A, B) + ((C0,) if C0 is not None else ()):
        if t.dim() != 3 or not t.is_cuda or t.stride(2) != 1:
            raise ValueError("operands: CUDA tensors [batch, rows, cols] with contiguous rows")
        if t.dtype != A.dtype or t.dtype not in (torch.complex64, torch.complex128):
            raise TypeError("complex64 or complex128 operands of one type")
    batch = A.shape[0]
    M = A.shape[2] if ta else A.shape[1]
    K = A.shape[1] if ta else A.shape[2]
    N = B.shape[1] if tb else B.shape[2]
    if (B.shape[2] if tb else B.shape[1]) != K or B.shape[0] != batch:
        raise ValueError("shapes do not chain")
    if out is None:
        out = torch.empty((batch, M, N), dtype=A.dtype, device=A.device)
    prec = FP32_REFINE if A.dtype == torch.complex64 else FP64
    c0p, ldc0, sc0 = (None, 0, 0) if C0 is None else (_dptr(C0), C0.stride(1), C0.stride(0))
    _check(lib().rci_cgemm_batched(M, N, K, int(ta), int(tb), float(alpha), _dptr(A), A.stride(1),
                                   A.stride(0), _dptr(B), B.stride(1), B.stride(0), float(beta),
                                   c0p, ldc0, sc0, _dptr(out), out.stride(1), out.stride(0), batch,
                                   prec, kernel, _stream(stream)))
    return out


def set_wait_limit(cycles: int) -> int:
    """Cycles a tensor-core pipeline wait may spin before its kernel gives up with
    RCI_ETIMEOUT (process-wide; <= 0 restores the default).  Returns the previous limit."""
    return int(lib().rci_set_wait_limit(int(cycles)))


def qform_toeplitz(v, lags, stream=None) -> float:
    """sum_{i,l} conj(v_i) lags[|i-l|] v_l on the device (v complex128, lags float64, CUDA)."""
    torch = _torch()
    v = v.to(torch.complex128).contiguous()
    lags = lags.to(torch.float64).contiguous()
    out = C.c_double()
    _check(lib().rci_qform_toeplitz(_dptr(v), _dptr(lags), v.numel(), C.byref(out),
                                    _stream(stream)))
    return out.value


QFORM_NOALLOC_MAX_N = 32768


def qform_toeplitz_noalloc(v, lags, out, stream=None):
    """Allocation-free form of qform_toeplitz for callers that must not allocate device
    memory: the result goes to the CUDA float64 tensor ``out`` (one element) in stream
    order, without synchronising.  n <= QFORM_NOALLOC_MAX_N."""
    torch = _torch()
    if v.dtype != torch.complex128 or lags.dtype != torch.float64 or out.dtype != torch.float64:
        raise TypeError("v complex128, lags and out float64")
    # the library receives raw device pointers: a host tensor, or one on another device than
    # the current one, would hand the kernel memory it cannot (or must not) address
    dev = torch.cuda.current_device()
    for name, t in (("v", v), ("lags", lags), ("out", out)):
        if not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device (cuda:{dev})")
    if not (v.is_contiguous() and lags.is_contiguous()):
        raise ValueError("contiguous tensors required")
    if lags.numel() < v.numel():
        raise ValueError("lags needs one entry per lag |i - l| < n (lags.numel() >= v.numel())")
    if out.numel() < 1:
        raise ValueError("out needs one element")
    _check(lib().rci_qform_toeplitz_noalloc(_dptr(v), _dptr(lags), v.numel(), _dptr(out),
                                            _stream(stream)))
    return out


def gauss_legendre(n: int, a: float = -1.0, b: float = 1.0, device: int = 0, stream=None):
    torch = _torch()
    x = torch.empty(n, dtype=torch.float64, device=torch.device("cuda", device))
    w = torch.empty_like(x)
    _check(lib().rci_gauss_legendre(n, a, b, _dptr(x), _dptr(w), _stream(stream)))
    return x, w


def grid_footprint(desc, prec=None, with_gradient: bool = False) -> int:
    """Device bytes of a grid for this descriptor (computed on the host)."""
    by = C.c_size_t()
    _check(lib().rci_grid_footprint(C.byref(_desc(desc, prec)), 1 if with_gradient else 0,
                                    C.byref(by)))
    return by.value


class Server:
    """Continuous-admission evaluation server on one device (see rci_server_* in rci.h).

    submit() returns a ticket at once; wait(ticket) returns the result as a dict (with the
    gradient as an array for gradient requests)."""

    def __init__(self, device: int = 0, slots: int = 4, arena_bytes: int = 0,
                 cache_bytes: int = 0, lookahead: int = 4):
        h = C.c_void_p()
        d = ServerDescC(device, slots, arena_bytes, cache_bytes, lookahead, 0)
        _check(lib().rci_server_create(C.byref(d), C.byref(h)))
        self._h = h
        self.device = device
        self._grads = {}

    def submit(self, desc, widths, obj, light, prec=None, want_grad: bool = False,
               design_key: int = 0) -> int:
        keep = []
        w = np.ascontiguousarray(np.asarray(widths, dtype=np.float64))
        grad = np.empty(w.size) if want_grad else None
        req = RequestC(_desc(desc, prec, self.device), _hptr(w), _objective(obj, keep),
                       _light(light, keep), 1 if want_grad else 0, 0, design_key,
                       _hptr(grad) if grad is not None else None)
        t = C.c_uint64()
        _check(lib().rci_server_submit(self._h, C.byref(req), C.byref(t)))
        self._grads[t.value] = grad      # written by the server before the ticket completes
        return t.value

    def wait(self, ticket: int, timeout: float = -1.0) -> dict:
        r = ResultC()
        _check(lib().rci_server_wait(self._h, ticket, timeout, C.byref(r)))
        grad = self._grads.pop(ticket, None)
        return {"status": r.status, "value": r.value, "cache_hit": bool(r.cache_hit),
                "refine_iters": r.refine_iters, "fp64_fallback": r.fp64_fallback,
                "simt_refactor": r.simt_refactor,
                "rel_residual": r.rel_residual,
                "t_submit_us": r.t_submit_us, "t_start_us": r.t_start_us,
                "t_end_us": r.t_end_us, "footprint": r.footprint, "grad": grad}

    def stats(self) -> dict:
        st = ServerStatsC()
        _check(lib().rci_server_stats_read(self._h, C.byref(st)))
        return {n: getattr(st, n) for n, _ in ServerStatsC._fields_ if n != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            lib().rci_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
