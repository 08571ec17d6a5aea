"""Host-side logic of the serving runtime (no GPU): the device footprint reported for a
grid against an independent count of its buffers, and the arena allocator against a
byte-ownership model (compiled with the host C++ compiler)."""
import math
import os
import shutil
import subprocess

import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _round(b):
    b = max(b, 16)
    return (b + 255) // 256 * 256


def _expected_footprint(d: W.GridDesc, fp64: bool, grad: bool) -> int:
    """Every buffer of a grid, from the layout: operator and vectors, BCR store, working
    arrays, level-0 factors, solve workspace (one right-hand side), gradient buffers."""
    nx = d.n_cells * d.cell_px + 2 * d.npml
    ny, ns = d.ny, d.n_cells * d.cell_px
    N, nn = nx * ny, ny * ny
    esz = 16 if fp64 else 8
    sizes = [8 * d.n_cells, 8 * N] + [16 * N] * 8
    sizes += [16 * N] if fp64 else [8 * N, 8 * N]
    T = math.ceil(ns / 128)
    sizes += [16 * ns, 16 * ns, 8 * ns, 8 * T * (T + 1) // 2, 64,
              8 * 1216 * 256, 8 * 1216 * 256, 8 * 256, 8 * (64 + 6 * 8192), 4]
    # block cyclic reduction levels
    n, m, off = [nx], [nx // 2], 0
    cur = (nx + 1) // 2
    while cur > 1:
        n.append(cur)
        m.append(cur // 2)
        off += 3 * (cur // 2) * nn
        cur = (cur + 1) // 2
    n.append(1)
    m.append(0)
    Lf = len(n) - 1
    m0, n1 = m[0], (nx + 1) // 2
    m0b = max(m0, 1) * ny
    sizes += [m0b * esz] * 4 + [m0b, m0b * ny * esz]
    sizes += [n1 * nn * esz] * 4 + [(off + nn) * esz, 4]
    ws = m0 * ny + sum(n[l] * ny for l in range(1, Lf + 1)) + \
        sum(m[l] * ny for l in range(1, Lf)) + 2 * (m[1] if Lf > 1 else 0) * ny + \
        2 * (m[2] if Lf > 2 else 0) * ny + ny
    sizes.append(ws * esz)
    if grad:
        sizes += [16 * N, 16 * ns, 16 * ns * math.ceil(ns / 1024), 8 * d.n_cells]
    return sum(_round(b) for b in sizes)


@pytest.mark.parametrize("shape", [(1, 96), (7, 100), (50, 128), (500, 160), (1250, 160), (2500, 224)])
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("grad", [False, True])
def test_footprint_matches_buffer_count(shape, fp64, grad):
    import paper_2207_10701_gb300 as P
    d = W.GridDesc(n_cells=shape[0], ny=shape[1])
    got = P.grid_footprint(d, prec=P.FP64 if fp64 else P.FP32_REFINE, with_gradient=grad)
    assert got == _expected_footprint(d, fp64, grad)


def test_footprint_rejects_bad_descriptor():
    import paper_2207_10701_gb300 as P
    with pytest.raises(P.RciError):
        P.grid_footprint(W.GridDesc(n_cells=0, ny=160))


def test_arena_allocator_against_model(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "arena_check")
    subprocess.run([cxx, "-O2", "-std=c++17", os.path.join(HERE, "native", "arena_check.cpp"),
                    "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and "arena ok" in out.stdout, out.stdout + out.stderr
