"""The serving runtime on the GPU: results in the mix equal results alone, admission by
device footprint, resident factorisations, overtaking within the look-ahead, and a
request that can never fit.

"Alone" is the plain API on a fresh grid (set_design, factor, avg_intensity[_grad]);
each served evaluation runs the same kernels on a grid of its own, so the two agree bit
for bit; a few requests are also checked against the oracle at the stated tolerances."""
import numpy as np
import pytest

import workloads as W
from oracle.reciprocal import Evaluation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2207_10701_gb300 as P  # noqa: E402

TOL = {P.FP64: 1e-9, P.FP32_REFINE: 1e-8}


def _alone(r, prec):
    with P.Grid(r.grid, prec=prec) as g:
        g.set_design(r.widths)
        g.factor()
        if r.want_grad:
            F, grad, _ = g.avg_intensity_grad(r.objective, r.light)
            return F, grad
        F, _ = g.avg_intensity(r.objective, r.light)
        return F, None


def _requests(n, seed, cells=(4, 40)):
    return W.serving_requests(n, 0.0, seed=seed, cells=cells, ny=96)


def test_mixed_requests_equal_alone_and_oracle():
    reqs = _requests(24, 3)
    precs = [P.FP32_REFINE if k % 3 else P.FP64 for k in range(len(reqs))]
    with P.Server(slots=4, arena_bytes=8 << 30, lookahead=4) as srv:
        tickets = [srv.submit(r.grid, r.widths, r.objective, r.light, prec=p, want_grad=r.want_grad)
                   for r, p in zip(reqs, precs)]
        res = [srv.wait(t, timeout=600) for t in tickets]
        st = srv.stats()
    assert st["submitted"] == st["completed"] == len(reqs) and st["failed"] == 0
    assert st["in_flight"] == 0 and st["queued"] == 0 and st["arena_used"] == 0
    for r, p, out in zip(reqs, precs, res):
        assert out["status"] == 0
        F, grad = _alone(r, p)
        assert out["value"] == F                       # bit for bit
        if r.want_grad:
            assert np.array_equal(out["grad"], grad)
        assert out["t_submit_us"] <= out["t_start_us"] <= out["t_end_us"]
    for k in (0, 1, 5):                                # and against the oracle
        r, p, out = reqs[k], precs[k], res[k]
        F_ref, _ = Evaluation(W.Workload("req", r.grid, r.objective, r.light, 0), r.widths).reciprocal()
        assert abs(out["value"] - F_ref) <= TOL[p] * abs(F_ref)


def test_resident_factorisation_is_reused():
    r = _requests(1, 8, cells=(30, 30))[0]
    other_light = W.Light(W.LIGHT_ANNULUS, th1=W.deg(12), th2=W.deg(27))
    with P.Server(slots=2, arena_bytes=4 << 30, cache_bytes=1 << 30) as srv:
        a = srv.wait(srv.submit(r.grid, r.widths, r.objective, r.light, design_key=77))
        b = srv.wait(srv.submit(r.grid, r.widths, r.objective, other_light, design_key=77))
        w2 = r.widths.copy()
        w2[0] += 0.01                                  # same key, different widths: no reuse
        c = srv.wait(srv.submit(r.grid, w2, r.objective, r.light, design_key=77))
        st = srv.stats()
    assert not a["cache_hit"] and b["cache_hit"] and not c["cache_hit"]
    assert st["cache_hits"] == 1 and st["resident"] >= 1
    r2 = W.Request(0.0, r.grid, r.widths, r.objective, other_light, False, 0)
    assert a["value"] == _alone(r, P.FP32_REFINE)[0]
    assert b["value"] == _alone(r2, P.FP32_REFINE)[0]


def test_admission_waits_for_memory_and_results_stay_exact():
    reqs = _requests(6, 11, cells=(60, 60))
    fp = P.grid_footprint(reqs[0].grid, prec=P.FP32_REFINE, with_gradient=True)
    with P.Server(slots=4, arena_bytes=int(1.6 * fp), lookahead=0) as srv:
        tickets = [srv.submit(r.grid, r.widths, r.objective, r.light, want_grad=r.want_grad)
                   for r in reqs]
        res = [srv.wait(t, timeout=600) for t in tickets]
        st = srv.stats()
    assert st["admission_waits"] >= 1 and st["arena_peak"] <= int(1.6 * fp)
    for r, out in zip(reqs, res):
        assert out["status"] == 0 and out["value"] == _alone(r, P.FP32_REFINE)[0]


def test_lookahead_lets_a_small_request_overtake():
    big = _requests(3, 21, cells=(200, 200))
    small = _requests(1, 22, cells=(5, 5))[0]
    fb = P.grid_footprint(big[0].grid, prec=P.FP32_REFINE, with_gradient=True)
    with P.Server(slots=3, arena_bytes=int(1.5 * fb), lookahead=4) as srv:
        t_big = [srv.submit(r.grid, r.widths, r.objective, r.light) for r in big]
        t_small = srv.submit(small.grid, small.widths, small.objective, small.light)
        out_small = srv.wait(t_small, timeout=600)
        outs = [srv.wait(t, timeout=600) for t in t_big]
        st = srv.stats()
    assert st["bypasses"] >= 1
    # the arena holds one big request at a time: the small one, submitted last, is admitted
    # while the second big one waits for the first (admission order, not execution speed;
    # the workers waiting for memory look at the queue again when a request arrives)
    assert out_small["t_start_us"] < outs[1]["t_start_us"]
    assert out_small["value"] == _alone(small, P.FP32_REFINE)[0]
    for r, out in zip(big, outs):
        assert out["status"] == 0 and out["value"] == _alone(r, P.FP32_REFINE)[0]


def test_request_larger_than_the_arena_fails_alone():
    big = _requests(1, 31, cells=(100, 100))[0]
    small = _requests(1, 32, cells=(4, 4))[0]
    fs = P.grid_footprint(small.grid, prec=P.FP32_REFINE, with_gradient=True)
    with P.Server(slots=2, arena_bytes=4 * fs) as srv:
        out_big = srv.wait(srv.submit(big.grid, big.widths, big.objective, big.light), timeout=600)
        out_small = srv.wait(srv.submit(small.grid, small.widths, small.objective, small.light),
                             timeout=600)
        with pytest.raises(P.RciError):
            srv.wait(123456)                          # unknown ticket
    assert out_big["status"] == 2                      # RCI_ENOMEM
    assert out_small["status"] == 0 and out_small["value"] == _alone(small, P.FP32_REFINE)[0]
