"""Host logic of the robust GRAPE loop (L-BFGS driver, masked slots, two-stage
validation, dJ ramp) with an oracle-backed stand-in for the GPU context."""
import numpy as np

import synth
from oracle import noise, robust


class OracleContext:
    def __init__(self, w, M, ins, tgs, mask):
        self.w, self.M, self.ins, self.tgs, self.mask = w, M, ins, tgs, mask
        self.u = None
        self.J = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass

    def set_controls(self, u):
        self.u = np.array(u, dtype=float)

    def sample_noise(self, seed, dist, scale):
        self.J = noise.sample_J(seed, self.M, self.w.N, dist, scale)

    def _pb(self):
        w = self.w
        return robust.Problem(N=w.N, K=w.K, dt=w.dt, C=w.C, chi=w.chi, u=self.u, mask=self.mask, J=self.J,
                              inputs=[m.sites for m in self.ins], targets=[m.sites for m in self.tgs])

    def fidelity_grad(self):
        F, g, _ = robust.ensemble(self._pb())
        return F, g

    def fidelity(self):
        F, _, _ = robust.ensemble(self._pb(), want_grad=False)
        return F


def test_grape_loop_with_oracle_context():
    from paper_2603_03639_gb300 import grape
    w = synth.WORKLOADS["x8"].replace(N=3, K=4, dt=0.25, M=3, P=2, chi=4)
    ins, tgs = w.states()
    mask = w.mask()
    mask[1, 0] = 0                                  # one masked slot must not move
    u0 = synth.pi_pulse_controls(w.K, w.C, w.N, w.dt)
    u0[:, 1, 0] = 0.123

    def make(M):
        return OracleContext(w, M, ins, tgs, mask)

    base = grape.validate(make, u0, w.M, (99, 0, 0.4))
    runs = grape.robust_ramp(make, u0, w.M, dJ_final=0.4, step=0.2, seed=3, mask=mask, maxiter=25)
    assert len(runs) == 2
    assert np.all(runs[-1].u[:, 1, 0] == 0.123)
    assert runs[-1].infidelity <= runs[-1].history[0] + 1e-15
    assert runs[-1].validation < base


def test_extend_controls_copies_sites_and_pairs():
    from paper_2603_03639_gb300 import grape
    rng = np.random.default_rng(0)
    u = rng.normal(size=(3, 3, 4))
    u[:, 2, 3] = 0.0                                 # the last site has no bond
    v = grape.extend_controls(u, 6, period=2)
    assert v.shape == (3, 3, 6)
    assert np.array_equal(v[:, :, :3], u[:, :, :3])
    assert np.array_equal(v[:, :2, 3], u[:, :2, 3])
    assert np.array_equal(v[:, 2, 3], u[:, 2, 1])    # the new bond (3, 4) copies bond (1, 2)
    assert np.array_equal(v[:, :, 4], v[:, :, 2]) and np.array_equal(v[:, :2, 5], v[:, :2, 3])
    assert np.all(v[:, 2, 5] == 0.0)
    w = grape.extend_controls(u[:, :2], 5, period=1)
    assert np.array_equal(w[:, :, 4], u[:, :2, 3])


def test_chain_ramp_with_oracle_context():
    from paper_2603_03639_gb300 import grape
    base = synth.WORKLOADS["x8"].replace(K=4, dt=0.25, P=2, chi=4)

    def make(n, M):
        w = base.replace(N=n)
        ins, tgs = w.states()
        return OracleContext(w, M, ins, tgs, w.mask())

    u2 = synth.controls(base.K, base.C, 2, 3, 0.5)
    runs = grape.chain_ramp(make, u2, [2, 3], lambda n: 2 * (n - 1), (4, 0, 0.2), maxiter=6)
    assert [r.u.shape[2] for r in runs] == [2, 3]
    assert all(r.validation is not None and 0.0 <= r.validation <= 1.0 for r in runs)
    assert runs[1].history[0] < 1.0


def test_served_objective_submits_and_waits():
    """ServedObjective turns each evaluation into a request to a serving loop
    (here a stand-in that evaluates with the oracle)."""
    import copy
    from paper_2603_03639_gb300 import grape
    from paper_2603_03639_gb300.serving import Request
    w = synth.WORKLOADS["x8"].replace(N=3, K=3, dt=0.25, M=2, P=2, chi=4)
    ins, tgs = w.states()
    ctx = OracleContext(w, w.M, ins, tgs, w.mask())

    class FakeServer:
        def __init__(self):
            self.seen = []

        def submit(self, req):
            self.seen.append(copy.copy(req))
            ctx.set_controls(req.controls)
            ctx.sample_noise(req.noise_seed, req.noise_dist, req.noise_scale)
            req.F, req.grad = ctx.fidelity_grad()
            req.finish = 1.0
            return req

        def wait(self, req):
            return req

    srv = FakeServer()
    tmpl = Request(key="x", N=w.N, K=w.K, dt=w.dt, chi=w.chi, M=w.M, C=w.C, inputs=ins, targets=tgs,
                   controls=np.zeros((w.K, w.C, w.N)), noise_seed=7, noise_dist=0, noise_scale=0.1)
    obj = grape.ServedObjective(srv, tmpl)
    u0 = synth.pi_pulse_controls(w.K, w.C, w.N, w.dt)
    r = grape.optimise_fn(obj, u0, maxiter=3)
    assert obj.requests == r.evaluations == len(srv.seen) > 0
    assert all(s.noise_seed == 7 and s.want_grad for s in srv.seen)
    assert r.infidelity <= r.history[0]
