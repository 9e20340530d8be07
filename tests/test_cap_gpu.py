"""Bonds at the cap chi_max = 64 on the GPU (Sec. II: the state is compressed
to a maximum bond size by truncated SVD).

The 14-qubit echo workload -- random controls, then the same controls
reversed in time and negated -- entangles the middle bonds past 64 at
mid-time, so theta reaches 128 x 128: the per-warp arrays at their largest,
theta and Phi in the warp's global scratch, the pivoted QR and the Jacobi
with 128-row columns, and cuts that the cap decides rather than the cutoff.
The echo then disentangles again, so the overlap with the input stays O(1)
and the 1e-10 bars are sharp.

Bars as everywhere: |dF| <= 1e-10, per-trajectory |dO| <= 1e-10, gradient
1e-8 relative.  Both sides also count the cap-decided cuts (forward and
costate updates) and their smallest relative gap (sigma_k - sigma_{k+1}) /
sigma_1, which must agree; a gap below 1e-10 would be reported as a tie at
the cut (the kept subspace then rests on rounding)."""
import numpy as np
import pytest

import synth
from oracle import robust
from tests._util import TOL_F, TOL_O, case, gpu_context, grad_close, oracle_problem

pytestmark = pytest.mark.gpu

TIE = 1e-10


def _report(tag, st_gpu, st_or):
    gap = st_gpu["min_trunc_gap"]
    print("%s: cap cuts gpu %d oracle %d; min relative gap gpu %.3e oracle %.3e%s"
          % (tag, st_gpu["cap_truncations"], st_or.get("cap_cuts", 0), gap, st_or.get("min_gap", -1.0),
             " (tie)" if 0.0 <= gap < TIE else ""))


def test_cap_decides_cuts_gradient_parity():
    w = synth.WORKLOADS["echo14"].replace(K=12, M=1, P=1)
    u, mask, J, ins, tgs = case(w)
    pb = oracle_problem(w, u, mask, J, ins, tgs)
    ctx = gpu_context(w, ins, tgs, mask)
    ctx.set_controls(u)
    ctx.set_noise(J)
    F, g = ctx.fidelity_grad()
    O = ctx.overlaps()
    st = ctx.stats()
    sto = {"discarded": 0.0, "dims": []}
    o, do = robust.trajectory(pb, 0, 0, want_grad=True, stats=sto)
    go = 2.0 * np.real(np.conj(o) * do)
    _report("echo14 K=12", st, sto)
    assert max(sto["dims"]) == 64 and st["max_bond"] == 64
    assert sto["cap_cuts"] > 0
    assert st["cap_truncations"] == sto["cap_cuts"]
    assert abs(st["min_trunc_gap"] - sto["min_gap"]) <= 1e-12
    assert abs(O[0, 0]) > 0.5
    assert abs(O[0, 0] - o) <= TOL_O
    assert abs(F - abs(o) ** 2) <= TOL_F
    assert grad_close(g, go)


def test_cap_overlaps_in_the_bench_launch_shape():
    """Forward only, two noise samples x two inputs (|0..0> and a random
    product state), the full 16 slices, in the launch shape bench.py uses
    for this workload."""
    from paper_2603_03639_gb300 import autotune
    w0 = synth.WORKLOADS["echo14"]
    warps, ctas = autotune.lookup(w0.N, w0.K, w0.chi, w0.M, w0.P, w0.C, grad=True)
    w = w0.replace(M=2, P=2)
    u, mask, J, ins, tgs = case(w)
    ctx = gpu_context(w, ins, tgs, mask, warps=warps, ctas_per_sm=ctas)
    ctx.set_controls(u)
    ctx.set_noise(J)
    F = ctx.fidelity()
    O = ctx.overlaps()
    st = ctx.stats()
    pb = oracle_problem(w, u, mask, J, ins, tgs)
    sto = {"discarded": 0.0, "dims": []}
    Fo = 0.0
    for s in range(w.M):
        for p in range(w.P):
            o, _ = robust.trajectory(pb, s, p, want_grad=False, stats=sto)
            assert abs(O[s, p] - o) <= TOL_O
            Fo += abs(o) ** 2 / (w.M * w.P)
    _report("echo14 M=2 P=2", st, sto)
    assert abs(F - Fo) <= TOL_F
    assert st["cap_truncations"] == sto["cap_cuts"] > 0
    assert abs(st["discarded_weight"] - sto["discarded"]) <= 1e-12 + 1e-6 * sto["discarded"]


def test_cap_operator_form_theta_128():
    """The operator form at chi = 32 (physical dimension 4, so theta is up to
    128 x 128 as well) with the cap deciding cuts, gradient included."""
    w = synth.WORKLOADS["cnotgate50"].replace(N=6, K=4, chi=32, M=1, P=1, dt=0.5, u_sigma=1.5, target="x",
                                              g_bonds="all")
    u, mask, J, ins, tgs = case(w)
    pb = oracle_problem(w, u, mask, J, ins, tgs)
    ctx = gpu_context(w, ins, tgs, mask)
    ctx.set_controls(u)
    ctx.set_noise(J)
    F, g = ctx.fidelity_grad()
    O = ctx.overlaps()
    st = ctx.stats()
    sto = {"discarded": 0.0, "dims": []}
    o, do = robust.trajectory(pb, 0, 0, want_grad=True, stats=sto)
    go = 2.0 * np.real(np.conj(o) * do)
    _report("operator N=6 chi=32", st, sto)
    assert max(sto["dims"]) == 32 and st["max_bond"] == 32
    assert st["cap_truncations"] == sto.get("cap_cuts", 0) > 0
    assert abs(O[0, 0] - o) <= TOL_O
    assert abs(F - abs(o) ** 2) <= TOL_F
    assert grad_close(g, go)
