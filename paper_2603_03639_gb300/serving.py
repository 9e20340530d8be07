"""Serving loop for many concurrent robust-GRAPE optimisers on one GPU.

Each request asks for F (and optionally dF/du) of one problem -- chain length,
chi_max, slices, ensemble, inputs/targets -- at one control vector, with its
own noise seed.  The server

  * keeps tnrc contexts resident on the device (canonical inputs/targets,
    gate tables, MPS and costate working slots) and reuses them for every
    later request of their problem, as an optimiser's iterations do; a
    request for a problem whose resident contexts are all busy gets another
    resident copy (made once, then reused like the first; at most max_copies
    per problem), so one problem can have several requests in flight;
  * admits a request when its context's device footprint fits the memory
    budget next to the contexts already holding work (idle contexts are
    destroyed first, least recently used, when memory is short);
  * launches every admitted request at once on its context's own CUDA
    stream, with the trajectory kernel in its pooled form (one CTA per
    trajectory, work regions from a pool), so requests that arrive while
    others run are admitted as slots and memory free up and their CTAs start
    as soon as any running trajectory ends (continuous batching at trajectory
    granularity); requests of problems that have been quick run on a
    high-priority stream, so the block scheduler starts their CTAs before the
    pending CTAs of long requests; pending requests are admitted shortest
    measured work first, and a short request even past the in-flight cap;
  * completes a request when its stream's event has fired, copying F and the
    gradient back, and records arrival, start and finish times.

Every evaluation is deterministic and independent of what else runs, so a
request's result is the same alone and in any mix.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Optional

import numpy as np

from .tnrc import Context, footprint


@dataclasses.dataclass
class Request:
    """One evaluation.  ``key`` identifies the problem (requests with equal
    keys share a resident context); inputs/targets are MPS objects (``pack()``)
    or (bond_dims, data) pairs."""
    key: str
    N: int
    K: int
    dt: float
    chi: int
    M: int
    C: int
    inputs: list
    targets: list
    controls: np.ndarray
    noise_seed: int
    noise_dist: int
    noise_scale: float
    want_grad: bool = True
    mask: Optional[np.ndarray] = None
    cutoff: float = 1e-12
    crosstalk: int = 1            # 1: ZZ; 3: J^x XX + J^y YY + J^z ZZ
    order: int = 2                # Trotter order (1: the slice of Eq. circuit)
    substeps: int = 1             # Trotter steps per control bin
    operator: bool = False        # evolve the operator from the identity (gate objective)
    # filled by the server
    priority: str = ""
    device_s: float = 0.0         # device span of the evaluation (CUDA events on its stream)
    arrival: float = 0.0
    start: float = 0.0
    finish: float = 0.0
    F: Optional[float] = None
    grad: Optional[np.ndarray] = None
    error: Optional[str] = None

    @property
    def P(self):
        return len(self.inputs)

    @property
    def latency(self):
        return self.finish - self.arrival

    def form(self):
        """Context keywords of the request's discretisation and form."""
        return {"crosstalk": self.crosstalk, "order": self.order, "substeps": self.substeps,
                "operator": self.operator}

    def footprint(self):
        return footprint(self.N, self.K, self.dt, self.chi, self.M, self.C, self.P, cutoff=self.cutoff,
                         mask=self.mask, **self.form())


class _Slot:
    """A resident context with its streams and device output buffers.

    The context launches its trajectories pooled (one CTA per trajectory),
    so the block scheduler can start other requests' CTAs whenever one of
    its trajectories ends; the slot owns a high- and a low-priority stream
    and runs each request on the one its problem's size calls for."""

    def __init__(self, req: Request, device):
        import torch
        self.key = req.key
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
        self.streams = (torch.cuda.Stream(device=device, priority=hi), torch.cuda.Stream(device=device, priority=lo))
        self.stream = self.streams[1]
        self.ctx = Context(req.N, req.K, req.dt, req.chi, req.M, req.C, req.inputs, req.targets,
                           cutoff=req.cutoff, mask=req.mask, stream=self.stream.cuda_stream, **req.form())
        self.ctx.set_pooled(True)   # other requests' CTAs can start between this one's trajectories
        self.ctx.set_graphs(True)   # each request replays the context's captured evaluation
        self.bytes = req.footprint()
        self.F = torch.zeros(1, dtype=torch.float64, device=device)
        self.g = torch.zeros((req.K, req.C, req.N), dtype=torch.float64, device=device)
        self.ev0 = torch.cuda.Event(enable_timing=True)
        self.event = torch.cuda.Event(enable_timing=True)
        self.busy: Optional[Request] = None
        self.last_used = 0.0
        self.service: Optional[float] = None   # shortest device span of this problem's requests (s)

    def launch(self, req: Request, high: bool):
        import torch
        st = self.streams[0] if high else self.streams[1]
        if st is not self.stream:
            self.ctx.set_stream(st.cuda_stream)
            self.stream = st
        with torch.cuda.stream(st):
            self.ev0.record(st)
            self.ctx.set_controls(req.controls)
            self.ctx.sample_noise(req.noise_seed, req.noise_dist, req.noise_scale)
            self.ctx.evaluate_dev(self.F.data_ptr(), self.g.data_ptr() if req.want_grad else 0)
            self.event.record(st)
        req.priority = "high" if high else "low"
        self.busy = req

    def collect(self):
        req = self.busy
        self.ctx.sync()
        span = self.ev0.elapsed_time(self.event) / 1000.0
        self.service = span if self.service is None else min(self.service, span)
        req.device_s = span
        req.F = float(self.F.item())
        req.grad = self.g.cpu().numpy().copy() if req.want_grad else None
        self.busy = None
        return req

    def close(self):
        self.ctx.close()


class Server:
    """Continuous-batching server on one device.

    mem_budget: device bytes the resident contexts may hold (default: 60% of
    the free memory at start); max_inflight: requests on the device at once
    (short requests may exceed it, up to four times);
    short_s: a request whose problem has been served in at most this many
    seconds of device time runs on a high-priority stream, so that its CTAs
    start before the pending CTAs of longer requests (shortest work first at
    trajectory granularity); a problem not yet measured runs at low priority;
    max_copies: resident contexts one problem may have, so that that many of
    its requests can be in flight at once (further ones wait for a copy to
    come free rather than for a new context to be built)."""

    def __init__(self, mem_budget: Optional[int] = None, max_inflight: int = 8, device: int = 0,
                 short_s: float = 0.1, max_copies: int = 2):
        import torch
        self.device = torch.device("cuda", device)
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            mem_budget = int(0.6 * free)
        self.mem_budget = mem_budget
        self.max_inflight = max_inflight
        self.short_s = short_s
        self.max_copies = max_copies
        self.key_service: dict = {}
        self.pending = collections.deque()
        self.slots: list = []
        self.done: list = []
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.stop = False
        self.admitted = 0
        self.peak_inflight = 0
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    # ---- client side ----
    def submit(self, req: Request) -> Request:
        req.arrival = time.perf_counter()
        with self.cv:
            self.pending.append(req)
            self.cv.notify()
        return req

    def wait(self, req: Request, timeout: float = 600.0) -> Request:
        """Block until ``req`` (submitted earlier) has finished or failed."""
        t0 = time.perf_counter()
        with self.cv:
            while req.finish == 0.0:
                if time.perf_counter() - t0 > timeout:
                    raise TimeoutError("request still pending")
                self.cv.wait(0.01)
        return req

    def drain(self, timeout: float = 600.0):
        """Wait until every submitted request has finished."""
        t0 = time.perf_counter()
        with self.cv:
            while self.pending or any(s.busy for s in self.slots):
                if time.perf_counter() - t0 > timeout:
                    raise TimeoutError("requests still pending")
                self.cv.wait(0.01)

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify()
        self.thread.join()
        for s in self.slots:
            s.close()
        self.slots = []

    # ---- server side ----
    def _drop(self, slot):
        """Release a failed slot's context now (its device memory stops
        counting towards the budget at the same moment)."""
        try:
            slot.close()
        except Exception:
            pass
        self.slots.remove(slot)

    def _service(self, key):
        """Shortest device span measured for this problem (s), or None; kept
        per problem, so that a new resident copy of it inherits the estimate."""
        known = [s.service for s in self.slots if s.key == key and s.service is not None]
        if known:
            self.key_service[key] = min(known + ([self.key_service[key]] if key in self.key_service else []))
        return self.key_service.get(key)

    def _admissible(self, req: Request) -> bool:
        """A resident copy of the request's problem is idle, or another copy
        may be made (at most max_copies per problem)."""
        mine = [s for s in self.slots if s.key == req.key]
        return any(s.busy is None for s in mine) or len(mine) < self.max_copies

    def _next_pending(self) -> Optional[Request]:
        """The pending request to admit next: among those whose problem has an
        idle resident copy (or may get one), the one whose problem has the
        shortest measured service time; unmeasured problems after measured
        ones; arrival order among equals."""
        best, best_t = None, None
        for r in self.pending:
            if not self._admissible(r):
                continue
            t = self._service(r.key)
            t = float("inf") if t is None else t
            if best is None or t < best_t:
                best, best_t = r, t
        return best

    def _held(self):
        return sum(s.bytes for s in self.slots)

    def _admit(self, req: Request) -> bool:
        idle = [s for s in self.slots if s.busy is None and s.key == req.key]
        if idle:
            slot = idle[0]
        else:
            need = req.footprint()
            if need > self.mem_budget:
                req.error = "request footprint %d B exceeds the server budget %d B" % (need, self.mem_budget)
                req.finish = time.perf_counter()
                self.done.append(req)
                return True
            # evict idle contexts of other problems, least recently used first
            while self._held() + need > self.mem_budget:
                idle_any = sorted((s for s in self.slots if s.busy is None), key=lambda s: s.last_used)
                if not idle_any:
                    return False
                victim = idle_any[0]
                victim.close()
                self.slots.remove(victim)
            import torch
            with torch.cuda.device(self.device):
                slot = _Slot(req, self.device)
            self.slots.append(slot)
        req.start = time.perf_counter()
        t = self._service(req.key)
        slot.launch(req, high=t is not None and t <= self.short_s)
        self.admitted += 1
        return True

    def _loop(self):
        import torch
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                if self.stop:
                    return
                # complete finished requests
                for s in list(self.slots):
                    if s.busy is not None and s.event.query():
                        req = s.busy
                        try:
                            s.collect()
                        except Exception as e:  # the context is unusable: drop it, fail the request
                            req.error = "evaluation failed: %s" % e
                            s.busy = None
                            self._drop(s)
                        req.finish = time.perf_counter()
                        s.last_used = req.finish
                        self.done.append(req)
                # admit while slots and memory allow, shortest known work first
                # (arrival order among equals): a short request does not wait
                # behind long ones for admission either
                inflight = sum(1 for s in self.slots if s.busy is not None)
                while self.pending:
                    req = self._next_pending()
                    if req is None:
                        break
                    t = self._service(req.key)
                    short = t is not None and t <= self.short_s
                    # a short request is admitted past the in-flight cap (up to
                    # four times it): its CTAs take SM slots as trajectories end
                    if inflight >= (4 * self.max_inflight if short else self.max_inflight):
                        break
                    try:
                        admitted = self._admit(req)
                    except Exception as e:  # creation or launch failed: fail this request only
                        req.error = "admission failed: %s" % e
                        req.finish = time.perf_counter()
                        self.done.append(req)
                        for s in [s for s in self.slots if s.busy is req]:
                            s.busy = None
                            self._drop(s)
                        admitted = True
                    if not admitted:
                        break
                    for i, r in enumerate(self.pending):   # by identity: requests hold arrays
                        if r is req:
                            del self.pending[i]
                            break
                    inflight = sum(1 for s in self.slots if s.busy is not None)
                self.peak_inflight = max(self.peak_inflight, inflight)
                self.cv.notify_all()
                if not self.pending and inflight == 0:
                    self.cv.wait(0.01)
            time.sleep(0.0002)


def latency_stats(reqs):
    """p50 / p99 latency (s) and throughput (requests/s) of finished requests."""
    lat = np.array([r.latency for r in reqs if r.error is None])
    if len(lat) == 0:
        return {"n": 0}
    span = max(r.finish for r in reqs) - min(r.arrival for r in reqs)
    return {"n": int(len(lat)), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "throughput_rps": len(lat) / span if span > 0 else None}
