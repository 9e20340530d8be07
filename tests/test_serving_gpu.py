"""Serving loop: requests of several problems arrive while others run; each
result must equal the one the same request gets alone."""
import numpy as np
import pytest

import synth
from oracle import noise

pytestmark = pytest.mark.gpu


def _requests(n, seed):
    from paper_2603_03639_gb300.serving import Request
    rng = np.random.default_rng(seed)
    shapes = [synth.WORKLOADS["x8"].replace(M=8, P=2),
              synth.WORKLOADS["x8"].replace(N=12, chi=16, K=10, M=4, P=2),
              synth.WORKLOADS["cnot50"].replace(N=20, chi=16, K=12, M=6, P=2),
              synth.WORKLOADS["ghz30"].replace(N=10, chi=8, K=15, M=5, P=1),
              synth.WORKLOADS["x8"].replace(M=4, P=2, order=1, substeps=2, crosstalk=3),
              synth.WORKLOADS["cnotgate50"].replace(N=8, chi=8, K=6, M=4)]
    states = [w.states() for w in shapes]
    reqs = []
    for i in range(n):
        j = int(rng.integers(len(shapes)))
        w = shapes[j]
        ins, tgs = states[j]
        reqs.append(Request(key="p%d" % j, N=w.N, K=w.K, dt=w.dt, chi=w.chi, M=w.M, C=w.C, inputs=ins,
                            targets=tgs, controls=rng.normal(0, 0.5, size=(w.K, w.C, w.N)),
                            noise_seed=int(rng.integers(1 << 40)), noise_dist=w.noise_dist,
                            noise_scale=w.noise_scale, want_grad=bool(i % 2 == 0), mask=w.mask(),
                            crosstalk=w.crosstalk, order=w.order, substeps=w.substeps, operator=w.operator))
    return reqs


def test_results_alone_equal_results_in_the_mix():
    import copy
    from paper_2603_03639_gb300.serving import Server, latency_stats
    reqs = _requests(16, 3)
    alone = [copy.copy(r) for r in reqs]
    srv = Server(max_inflight=1)
    for r in alone:
        srv.submit(r)
        srv.drain()
    srv.close()
    mix = [copy.copy(r) for r in reqs]
    srv = Server(max_inflight=8)
    for r in mix:
        srv.submit(r)
    srv.drain()
    peak = srv.peak_inflight
    srv.close()
    assert peak > 1
    for a, b in zip(alone, mix):
        assert a.error is None and b.error is None
        assert a.F == b.F
        if a.want_grad:
            assert np.array_equal(a.grad, b.grad)
    st = latency_stats(mix)
    assert st["n"] == len(mix) and st["p99_s"] >= st["p50_s"] > 0


def test_request_larger_than_budget_is_refused_and_server_keeps_going():
    from paper_2603_03639_gb300.serving import Server
    reqs = _requests(3, 4)
    big = reqs[0]
    srv = Server(mem_budget=big.footprint() - 1, max_inflight=4)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    srv.close()
    errs = [r for r in reqs if r.error]
    assert big in errs
    assert all(r.F is not None for r in reqs if r.footprint() < big.footprint())


def test_short_request_overtakes_a_long_one():
    """Continuous batching at trajectory granularity: a short request that
    arrives while a long one occupies every SM finishes first -- its CTAs
    (high-priority stream) start as soon as some of the long request's
    trajectories end, instead of after the whole long request."""
    import time
    from paper_2603_03639_gb300.serving import Request, Server
    rng = np.random.default_rng(9)

    def req(w, key):
        ins, tgs = w.states()
        return Request(key=key, N=w.N, K=w.K, dt=w.dt, chi=w.chi, M=w.M, C=w.C, inputs=ins, targets=tgs,
                       controls=rng.normal(0, 0.5, size=(w.K, w.C, w.N)), noise_seed=int(rng.integers(1 << 40)),
                       noise_dist=w.noise_dist, noise_scale=w.noise_scale, want_grad=True, mask=w.mask())

    long_w = synth.WORKLOADS["x50"].replace(M=96)
    short_w = synth.WORKLOADS["x8"].replace(M=8)
    srv = Server(max_inflight=4)
    for w, key in ((long_w, "long"), (short_w, "short")):   # resident and measured
        srv.submit(req(w, key))
        srv.drain()
    big = srv.submit(req(long_w, "long"))
    time.sleep(0.05)
    small = srv.submit(req(short_w, "short"))
    srv.drain()
    srv.close()
    assert big.error is None and small.error is None
    assert small.priority == "high" and big.priority == "low"
    assert small.finish < big.finish
