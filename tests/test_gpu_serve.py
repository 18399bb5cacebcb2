"""Serving loop: results against the oracle, the same bits alone and in the
mix, admission under a memory cap, and overlap of requests on the device."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2308_00106_gb300 import maxe
from paper_2308_00106_gb300 import serve
from paper_2308_00106_gb300 import workloads as W
from tests.gpu_common import code, rel_l2

pytestmark = pytest.mark.gpu


def _mats():
    return [W.poisson_uniform(500 + m, rows, lam, "f32" if m % 2 == 0 else "bf16", device="cuda")
            for m, (rows, lam) in enumerate([(2000, 5.0), (9000, 20.0), (30000, 12.0), (4000, 45.0),
                                             (60000, 8.0), (15000, 30.0)])]


@pytest.fixture(scope="module")
def server():
    maxe.load(build_if_missing=True)
    srv = serve.Server(_mats(), seed=77, mem_cap_bytes=8 << 30)
    yield srv
    srv.close()
    torch.cuda.synchronize()
    assert maxe.maxe_device_status() == maxe.MAXE_OK


@pytest.fixture(scope="module")
def server_xs():
    """Every handle with the x-sliced form: SpMV products go out as single x-sliced launches."""
    maxe.load(build_if_missing=True)
    srv = serve.Server(_mats(), seed=77, mem_cap_bytes=8 << 30, xslice=True)
    assert all(h.xslice() for h in srv.handles)
    yield srv
    srv.close()
    torch.cuda.synchronize()
    assert maxe.maxe_device_status() == maxe.MAXE_OK


@pytest.fixture(params=["autotuned", "xsliced"])
def any_server(request, server, server_xs):
    return server if request.param == "autotuned" else server_xs


def _check(srv, r):
    A = srv.mats[r.mat].to("cpu")
    h = srv.handles[r.mat]
    nrp, nco, nva, rperm, cperm = h.csr()
    v = nva.cpu()
    vv = v.view(torch.int16).numpy().view(np.uint16) if v.dtype == torch.bfloat16 else v.numpy()
    if r.kind == "power":
        lam, u, u0 = r.result
        v0 = np.empty(A.cols)
        v0[cperm.cpu().numpy()] = u0.cpu().double().numpy()  # original-space start vector
        rp, co, va = A.numpy()
        lo, vo = oracle.power_iteration(A.rows, rp, co, va, code(A.dtype), v0, r.steps)
        assert lam == pytest.approx(lo, rel=1e-4)
    else:
        g = torch.Generator(device="cuda")
        g.manual_seed(r.seed)
        X = (torch.rand(A.cols, r.k, generator=g, device="cuda") * 2 - 1).cpu().double().numpy()
        ref = oracle.spmm(A.rows, nrp.cpu().numpy(), nco.cpu().numpy(), vv, code(A.dtype), X)
        assert rel_l2(r.result.cpu().numpy(), ref) <= 1e-5


def test_serving_results_match_oracle(any_server):
    server = any_server
    trace = serve.make_trace(40, len(server.mats), math.inf, seed=3, mix=(0.4, 0.4, 0.2), kmax=8, steps=6)
    stats = server.run(trace, keep_results=True)
    assert stats["requests"] == 40 and stats["max_batch"] > 1
    for r in trace:
        _check(server, r)


def test_serving_same_alone_and_in_mix(any_server):
    server = any_server
    trace = serve.make_trace(30, len(server.mats), 4000.0, seed=9, mix=(0.4, 0.4, 0.2), kmax=8, steps=5)
    server.run(trace, keep_results=True)
    for r in trace:
        alone = serve.clone_request(r)
        server.run([alone], keep_results=True)
        if r.kind == "power":
            assert alone.result[0] == r.result[0]
            assert torch.equal(alone.result[1], r.result[1])
        else:
            assert torch.equal(alone.result, r.result)


def test_admission_respects_memory_cap(server):
    trace = serve.make_trace(24, len(server.mats), math.inf, seed=5, mix=(0.0, 1.0, 0.0), kmax=32)
    need = max(server.request_bytes(r) for r in trace)
    old = server.mem_cap
    server.mem_cap = server.resident_bytes + 2 * need  # room for about two requests at a time
    try:
        stats = server.run(trace)
    finally:
        server.mem_cap = old
    assert stats["requests"] == 24
    assert stats["peak_request_bytes"] <= 2 * need


def test_requests_overlap_on_device(server):
    """Continuous batching: with all requests queued, steps carry several requests."""
    trace = serve.make_trace(50, len(server.mats), math.inf, seed=1)
    stats = server.run(trace)
    assert stats["max_batch"] >= 10 and stats["batch_steps"] < 50 * 3
