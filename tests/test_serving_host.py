"""Host-side policy of the serving loop, on the CPU: which pending request is
admitted next, when a problem may take another resident copy, how the
per-problem service estimate is kept, and the latency statistics.  The
server object is built without its device thread; its slots are stand-ins
that carry only what the policy reads (problem key, busy request, measured
service time)."""
import collections

import numpy as np

from paper_2603_03639_gb300.serving import Request, Server, latency_stats


class Slot:
    def __init__(self, key, busy=None, service=None):
        self.key, self.busy, self.service = key, busy, service


def server(slots, max_copies=2):
    s = object.__new__(Server)   # no device, no thread: the policy methods only
    s.slots = list(slots)
    s.max_copies = max_copies
    s.key_service = {}
    s.pending = collections.deque()
    s.short_s = 0.1
    return s


def request(key, arrival=0.0, finish=0.0, error=None):
    r = Request(key=key, N=4, K=2, dt=0.1, chi=4, M=1, C=3, inputs=[], targets=[],
                controls=np.zeros((2, 3, 4)), noise_seed=1, noise_dist=0, noise_scale=0.0)
    r.arrival, r.finish, r.error = arrival, finish, error
    return r


def test_shortest_measured_problem_first_then_unmeasured_in_arrival_order():
    s = server([Slot("slow", service=0.5), Slot("fast", service=0.01)])
    a, b, c, d = request("slow"), request("fast"), request("new1"), request("new2")
    s.pending.extend([c, a, d, b])
    order = []
    while s.pending:
        r = s._next_pending()
        order.append(r)
        s.pending = collections.deque(x for x in s.pending if x is not r)   # by identity, as the server does
    assert [r.key for r in order] == ["fast", "slow", "new1", "new2"]


def test_equal_problems_keep_arrival_order():
    s = server([Slot("p", service=0.2)])
    first, second = request("p"), request("p")
    s.pending.extend([first, second])
    assert s._next_pending() is first


def test_copies_per_problem():
    busy = request("p")
    # one busy copy: a second copy may be made
    assert server([Slot("p", busy=busy)])._admissible(request("p"))
    # two busy copies at max_copies = 2: the request waits
    assert not server([Slot("p", busy=busy), Slot("p", busy=busy)])._admissible(request("p"))
    # an idle copy serves it whatever the count
    assert server([Slot("p", busy=busy), Slot("p")])._admissible(request("p"))
    # max_copies = 1 and the only copy busy: wait
    assert not server([Slot("p", busy=busy)], max_copies=1)._admissible(request("p"))
    # other problems' copies do not count
    assert server([Slot("q", busy=busy), Slot("q", busy=busy)])._admissible(request("p"))


def test_a_waiting_problem_does_not_block_the_others():
    busy = request("p")
    s = server([Slot("p", busy=busy, service=0.01), Slot("p", busy=busy, service=0.01), Slot("q", service=0.9)])
    s.pending.extend([request("p"), request("q")])
    assert s._next_pending().key == "q"   # p is shorter but has no free copy


def test_service_estimate_is_the_shortest_span_and_outlives_its_slot():
    s = server([Slot("p", service=0.3), Slot("p", service=0.2), Slot("q")])
    assert s._service("p") == 0.2
    assert s._service("q") is None
    s.slots = [Slot("p", service=0.25)]     # the faster copy was evicted, a new one measured
    assert s._service("p") == 0.2
    s.slots = []
    assert s._service("p") == 0.2


def test_latency_stats():
    lat = np.array([0.01, 0.02, 0.03, 0.04, 1.0])
    reqs = [request("p", arrival=1.0 + i, finish=1.0 + i + x) for i, x in enumerate(lat)]
    reqs.append(request("p", arrival=0.5, finish=9.0, error="admission failed"))
    st = latency_stats(reqs)
    assert st["n"] == 5
    assert abs(st["p50_s"] - 0.03) < 1e-12
    assert abs(st["p99_s"] - np.percentile(lat, 99)) < 1e-12
    assert abs(st["mean_s"] - lat.mean()) < 1e-12
    # the span runs from the first arrival to the last finish, failed requests included
    assert abs(st["throughput_rps"] - 5 / (9.0 - 0.5)) < 1e-12
    assert latency_stats([request("p", error="x")]) == {"n": 0}
