"""The seeded input recipe (no GPU): sizes of the named workloads, the width distribution,
determinism under a seed, and the statistics of the serving request stream."""
import math

import numpy as np
import pytest

import workloads as W


def _nx(g):
    return g.n_cells * g.cell_px + 2 * g.npml


@pytest.mark.parametrize("make, nx, ny", [(W.c1_concentrator, 440, 128), (W.c2_collimator, 4040, 160),
                                          (W.c3_precision, 20040, 224), (W.c4_gradient, 4040, 160)])
def test_named_workload_sizes(make, nx, ny):
    wl = make()
    assert _nx(wl.grid) == nx and wl.grid.ny == ny
    # width of the metasurface in wavelengths: cells x period
    assert wl.grid.n_cells * wl.grid.cell_px / wl.grid.ppl == pytest.approx((nx - 2 * wl.grid.npml) / wl.grid.ppl)


def test_widths_are_seeded_uniform_in_range():
    a, b = W.widths(5000, 7), W.widths(5000, 7)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, W.widths(5000, 8))
    assert a.min() >= 0.08 and a.max() <= 0.36
    # uniform on [0.08, 0.36]: mean 0.22, variance 0.28^2 / 12
    assert a.mean() == pytest.approx(0.22, abs=0.004)
    assert a.var() == pytest.approx(0.28 ** 2 / 12, rel=0.05)


def test_collimator_light_and_objective():
    wl = W.c2_collimator()
    assert wl.light.kind == W.LIGHT_ANNULUS
    assert wl.light.th1 == pytest.approx(math.radians(10)) and wl.light.th2 == pytest.approx(math.radians(30))
    assert wl.objective.kind == W.OBJ_PLANEWAVE and wl.objective.theta_out == 0.0
    assert wl.n_angles == 1000


def test_serving_stream_statistics():
    n, rate = 4096, 50.0
    reqs = W.serving_requests(n, rate, seed=3)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) >= 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(1 / rate, rel=0.05)          # exponential, mean 1/rate
    assert np.std(gaps) == pytest.approx(1 / rate, rel=0.08)         # and std 1/rate
    cells = np.array([r.grid.n_cells for r in reqs])
    assert cells.min() >= 50 and cells.max() <= 1250
    # log-uniform in cells: the median sits at the geometric mean
    assert np.median(cells) == pytest.approx(math.sqrt(50 * 1250), rel=0.08)
    grad = np.mean([r.want_grad for r in reqs])
    assert grad == pytest.approx(0.3, abs=0.03)
    kinds = np.mean([r.objective.kind == W.OBJ_VIRTUAL_FOCUS for r in reqs])
    assert kinds == pytest.approx(0.5, abs=0.03)
    for r in reqs[:200]:
        assert len(r.widths) == r.grid.n_cells and r.grid.ny == 160
        if r.light.kind == W.LIGHT_CONE:
            assert math.radians(5) <= r.light.c <= math.radians(40)
        else:
            assert math.radians(5) <= r.light.th1 < r.light.th2 <= math.radians(40)


def test_serving_stream_is_deterministic_and_designs_distinct():
    a, b = W.serving_requests(64, 10.0, seed=5), W.serving_requests(64, 10.0, seed=5)
    assert [r.arrival_s for r in a] == [r.arrival_s for r in b]
    assert all(np.array_equal(x.widths, y.widths) for x, y in zip(a, b))
    assert len({r.seed for r in a}) == 64
    c = W.serving_requests(64, 10.0, seed=6)
    assert not set(r.seed for r in a) & set(r.seed for r in c)
