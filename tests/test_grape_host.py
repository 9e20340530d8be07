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
