"""Host logic of the serving workload (CPU): the request traces the serving
benchmark replays -- Poisson arrivals, the request mix, SpMM widths and
power-iteration lengths -- and the unit accounting the server admits by."""
import math

import numpy as np

from paper_2308_00106_gb300 import serve


def test_trace_is_seeded_and_sorted():
    a = serve.make_trace(500, 7, 200.0, seed=3)
    b = serve.make_trace(500, 7, 200.0, seed=3)
    assert [(r.arrival, r.mat, r.kind, r.k, r.steps, r.seed) for r in a] == \
           [(r.arrival, r.mat, r.kind, r.k, r.steps, r.seed) for r in b]
    t = np.array([r.arrival for r in a])
    assert (np.diff(t) >= 0).all() and t[0] > 0
    assert [r.rid for r in a] == list(range(500))
    assert len({r.seed for r in a}) == 500
    c = serve.make_trace(500, 7, 200.0, seed=4)
    assert [r.mat for r in a] != [r.mat for r in c]


def test_poisson_arrival_rate():
    """Exponential gaps: mean 1/rate, and the coefficient of variation of an
    exponential law is 1."""
    rate = 1000.0
    t = np.array([r.arrival for r in serve.make_trace(20000, 4, rate, seed=1)])
    gaps = np.diff(np.r_[0.0, t])
    assert abs(gaps.mean() * rate - 1.0) < 0.03
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05


def test_saturation_trace_arrives_at_once():
    tr = serve.make_trace(100, 3, math.inf, seed=2)
    assert all(r.arrival == 0.0 for r in tr)


def test_request_mix_widths_and_units():
    n, kmax, steps = 30000, 32, 20
    tr = serve.make_trace(n, 64, 50.0, seed=5, mix=(0.6, 0.3, 0.1), kmax=kmax, steps=steps)
    kinds = np.array([r.kind for r in tr])
    for kind, p in (("spmv", 0.6), ("spmm", 0.3), ("power", 0.1)):
        frac = (kinds == kind).mean()
        assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / n), (kind, frac)
    mats = np.array([r.mat for r in tr])
    assert mats.min() == 0 and mats.max() == 63
    for r in tr:
        if r.kind == "spmm":
            assert 2 <= r.k <= kmax and r.steps == 0 and r.units == 1
        elif r.kind == "power":
            assert r.k == 1 and r.steps == steps and r.units == steps + 1
        else:
            assert r.k == 1 and r.steps == 0 and r.units == 1
    ks = np.array([r.k for r in tr if r.kind == "spmm"])
    assert set(np.unique(ks)) == set(range(2, kmax + 1))


def test_clone_keeps_the_work_and_resets_the_timeline():
    r = serve.make_trace(3, 5, 10.0, seed=9)[2]
    r.t_admit, r.t_done, r.units_done = 1.0, 2.0, 3
    c = serve.clone_request(r, arrival=0.5)
    assert (c.rid, c.mat, c.kind, c.k, c.steps, c.seed) == (r.rid, r.mat, r.kind, r.k, r.steps, r.seed)
    assert c.arrival == 0.5 and math.isnan(c.t_admit) and math.isnan(c.t_done) and c.units_done == 0
    c.t_done = 0.75
    assert abs(c.latency - 0.25) < 1e-15
