"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/rci.h declares (no device calls; runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rci.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"\b(rci_[a-z_0-9]+)\s*\(", txt))


@pytest.fixture(scope="module")
def libpath():
    from paper_2207_10701_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    declared = _declared()
    assert declared, "no declarations parsed"
    assert declared <= exported, declared - exported


def test_binding_covers_header_and_loads(libpath):
    import paper_2207_10701_gb300 as P
    L = P.lib(libpath)
    assert set(P.EXPORTED) == _declared()
    assert L.rci_status_str(5).decode() == "singular diagonal block"
    assert L.rci_status_str(0).decode() == "ok"


def test_library_is_built_for_sm103a_only(libpath):
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    arches = set(re.findall(r"sm_\d+a?", out.stdout))
    assert arches == {"sm_103a"}, arches


def test_invalid_descriptor_is_rejected_without_a_device(libpath):
    import ctypes as C
    import paper_2207_10701_gb300.rci as R
    import workloads as W
    d = R._desc(W.GridDesc(n_cells=2, ny=8))      # ny too small for PML + layers
    h = C.c_void_p()
    assert R.lib().rci_create_grid(C.byref(d), None, C.byref(h)) == 1   # RCI_EINVAL
    assert R.lib().rci_qform_toeplitz(None, None, 0, None, None) == 1


def test_descriptor_limits_of_the_solver_are_checked_at_creation(libpath):
    # the footprint query validates a descriptor exactly as grid creation does, on the host
    import ctypes as C
    import paper_2207_10701_gb300.rci as R
    import workloads as W

    def footprint(ny, prec):
        d = R._desc(W.GridDesc(n_cells=2, ny=ny, prec=prec))
        b = C.c_size_t()
        return R.lib().rci_grid_footprint(C.byref(d), 0, C.byref(b))

    assert footprint(256, R.FP64) == 0 and footprint(256, R.FP32_REFINE) == 0
    assert footprint(258, R.FP64) == 1 and footprint(258, R.FP32_REFINE) == 1   # RCI_EINVAL
    assert footprint(161, R.FP64) == 0
    assert footprint(161, R.FP32_REFINE) == 1      # FP32 rows are read as complex64 pairs
