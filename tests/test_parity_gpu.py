"""GPU (C ABI) against the oracle on the same seeded inputs.

Bars: |F_gpu - F_oracle| <= 1e-10, ||g_gpu - g_oracle|| <= 1e-8 ||g_oracle||
(and per component against the largest component), per-trajectory overlaps
to 1e-10; noise draws bit-exact (uniform) or to 1e-15 relative (normal)."""
import numpy as np
import pytest

import synth
from oracle import noise, robust
from tests._util import TOL_F, TOL_O, case, gpu_context, grad_close, oracle_problem

pytestmark = pytest.mark.gpu


def run_both(w, u=None, grad=True, g_fixed=None, checkpoint_every=0, pairs=None):
    u, mask, J, ins, tgs = case(w, u)
    pb = oracle_problem(w, u, mask, J, ins, tgs, g_fixed)
    ctx = gpu_context(w, ins, tgs, mask, g_fixed, checkpoint_every)
    ctx.set_controls(u)
    ctx.set_noise(J)
    if grad:
        F, g = ctx.fidelity_grad()
    else:
        F = ctx.fidelity()
        g = None
    O = ctx.overlaps()
    Fo, go, Oo = robust.ensemble(pb, want_grad=grad, pairs=pairs)
    return ctx, (F, g, O), (Fo, go, Oo)


def test_x8_fidelity_all_trajectories():
    w = synth.WORKLOADS["x8"]
    ctx, (F, _, O), (Fo, _, Oo) = run_both(w, grad=False)
    assert abs(F - Fo) <= TOL_F
    assert np.max(np.abs(O - Oo)) <= TOL_O
    st = ctx.stats()
    assert st["max_bond"] <= 16 and sum(st["bond_hist"]) > 0


def test_x8_gradient_random_controls():
    w = synth.WORKLOADS["x8"].replace(M=4)
    _, (F, g, O), (Fo, go, Oo) = run_both(w)
    assert abs(F - Fo) <= TOL_F
    assert np.max(np.abs(O - Oo)) <= TOL_O
    assert grad_close(g, go)


def test_x8_near_solution_high_fidelity():
    w = synth.WORKLOADS["x8"].replace(M=4, noise_scale=0.05)
    u = synth.pi_pulse_controls(w.K, w.C, w.N, w.dt, seed=5, jitter=0.05)
    _, (F, g, O), (Fo, go, Oo) = run_both(w, u=u)
    assert Fo > 0.5
    assert abs(F - Fo) <= TOL_F
    assert grad_close(g, go)


@pytest.mark.parametrize("N", [2, 3, 5])
def test_short_chains_and_odd_lengths(N):
    w = synth.WORKLOADS["x8"].replace(N=N, K=3, M=2, P=2, chi=4)
    _, (F, g, O), (Fo, go, Oo) = run_both(w)
    assert abs(F - Fo) <= TOL_F
    assert grad_close(g, go)


def test_cnot_layout_masked_g_and_fixed_zz():
    w = synth.WORKLOADS["cnot50"].replace(N=8, K=6, chi=16, M=3, P=2)
    rng = np.random.default_rng(3)
    gfix = rng.normal(0, 0.2, size=(w.K, w.N - 1))
    _, (F, g, O), (Fo, go, Oo) = run_both(w, g_fixed=gfix)
    assert abs(F - Fo) <= TOL_F
    assert grad_close(g, go)
    assert np.all(g[:, 2, 1::2] == 0.0)


def test_truncated_regime_and_large_theta():
    # strong controls on 12 sites: bond dims reach the cap; theta up to 64 x 64
    w = synth.WORKLOADS["ghz30"].replace(N=12, K=5, chi=32, M=1, P=1, u_sigma=1.5, dt=0.25)
    _, (F, g, O), (Fo, go, Oo) = run_both(w)
    assert abs(F - Fo) <= TOL_F
    assert np.max(np.abs(O - Oo)) <= TOL_O
    assert grad_close(g, go)


def test_hard_truncation_chi_4():
    w = synth.WORKLOADS["ghz30"].replace(N=10, K=4, chi=4, M=2, P=1, u_sigma=1.0, dt=0.2)
    _, (F, g, O), (Fo, go, Oo) = run_both(w)
    assert abs(F - Fo) <= TOL_F
    assert grad_close(g, go)


@pytest.mark.parametrize("shape", [(8, 1), (4, 2), (2, 4), (8, 2), (4, 4)])
def test_launch_shapes_and_register_builds(shape):
    """Every launch shape -- including more than 8 warps per SM, which runs the
    128-register build of the trajectory kernel -- meets the oracle bars, on a
    case with small thetas (shared slabs) and one with 64 x 64 thetas (global
    scratch)."""
    warps, ctas = shape
    for w in (synth.WORKLOADS["x8"].replace(M=4),
              synth.WORKLOADS["ghz30"].replace(N=12, K=5, chi=32, M=1, P=1, u_sigma=1.5, dt=0.25)):
        u, mask, J, ins, tgs = case(w)
        pb = oracle_problem(w, u, mask, J, ins, tgs)
        ctx = gpu_context(w, ins, tgs, mask, warps=warps, ctas_per_sm=ctas)
        ctx.set_controls(u)
        ctx.set_noise(J)
        F, g = ctx.fidelity_grad()
        Fo, go, Oo = robust.ensemble(pb, want_grad=True)
        assert abs(F - Fo) <= TOL_F
        assert np.max(np.abs(ctx.overlaps() - Oo)) <= TOL_O
        assert grad_close(g, go)


@pytest.mark.parametrize("name,order,substeps,N,P", [("cnot50", 1, 1, 8, 2), ("ghz30", 1, 2, 7, 1),
                                                      ("cnot50", 2, 3, 8, 2), ("x8", 1, 1, 2, 2),
                                                      ("x8", 1, 3, 5, 2), ("x8", 2, 2, 6, 2)])
def test_trotter_order_and_substeps(name, order, substeps, N, P):
    """The first-order slice of Eq. circuit (rotations folded into the bond
    gates) and several Trotter steps per control bin, against the oracle."""
    w = synth.WORKLOADS[name].replace(N=N, K=4, chi=16, M=2, P=P, order=order, substeps=substeps)
    _, (F, g, O), (Fo, go, Oo) = run_both(w)
    assert abs(F - Fo) <= TOL_F
    assert np.max(np.abs(O - Oo)) <= TOL_O
    assert grad_close(g, go)


def test_first_order_heisenberg_crosstalk_truncated():
    w = synth.WORKLOADS["ghz30"].replace(N=10, K=5, chi=8, M=2, P=1, u_sigma=1.0, dt=0.2, order=1, substeps=2,
                                         crosstalk=3)
    _, (F, g, O), (Fo, go, Oo) = run_both(w)
    assert abs(F - Fo) <= TOL_F
    assert grad_close(g, go)


@pytest.mark.parametrize("target,order,terms,N,chi", [("cnot", 2, 1, 8, 16), ("x", 2, 3, 7, 16), ("cnot", 1, 3, 8, 16),
                                                      ("cnot", 2, 1, 10, 4), ("x", 1, 1, 5, 8)])
def test_operator_form_parity(target, order, terms, N, chi):
    """The MPO of Sec. II (operators as vectors, physical dimension 4) from the
    identity: the gate fidelity |tr(U_T^dag U) / 2^N|^2 of Eq. gateinfid, its
    gradient and the per-sample overlaps against the oracle, untruncated and
    truncated (chi = 4)."""
    w = synth.WORKLOADS["cnotgate50"].replace(N=N, K=4, chi=chi, M=3, P=1, target=target, order=order,
                                              crosstalk=terms, g_bonds="pairs" if target == "cnot" else "all")
    # near the pi pulse the X-gate fidelity is O(1) (random controls give ~0)
    u = synth.pi_pulse_controls(w.K, w.C, w.N, w.dt, seed=5, jitter=0.1) if target == "x" else None
    _, (F, g, O), (Fo, go, Oo) = run_both(w, u=u)
    assert abs(F - Fo) <= TOL_F
    assert np.max(np.abs(O - Oo)) <= TOL_O
    assert grad_close(g, go)


def test_checkpoint_segments_do_not_change_results(monkeypatch):
    """Checkpoint/recompute segmentations (history cap 0 forces that path) and
    the packed history give bitwise the same result."""
    w = synth.WORKLOADS["x8"].replace(K=7, M=2, P=2)
    u, mask, J, ins, tgs = case(w)
    res = []
    ctx = gpu_context(w, ins, tgs, mask)
    ctx.set_controls(u)
    ctx.set_noise(J)
    res.append(ctx.fidelity_grad())
    monkeypatch.setenv("TNRC_HISTORY_CAP", "0")
    for ce in (1, 3, 7, 0):
        ctx = gpu_context(w, ins, tgs, mask, checkpoint_every=ce)
        ctx.set_controls(u)
        ctx.set_noise(J)
        res.append(ctx.fidelity_grad())
    for F, g in res[1:]:
        assert F == res[0][0] and np.array_equal(g, res[0][1])


def test_heisenberg_crosstalk_parity():
    """The general parasitic model of Eq. Hp: J^x XX + J^y YY + J^z ZZ per bond."""
    w = synth.WORKLOADS["cnot50"].replace(N=8, K=6, chi=16, M=3, P=2, crosstalk=3, noise_dist=0, noise_scale=0.2)
    _, (F, g, O), (Fo, go, Oo) = run_both(w)
    assert abs(F - Fo) <= TOL_F
    assert np.max(np.abs(O - Oo)) <= TOL_O
    assert grad_close(g, go)


@pytest.mark.parametrize("terms", [1, 3])
def test_device_noise_matches_oracle_generator(terms):
    for dist, scale in ((0, 0.1), (1, 0.05)):
        w = synth.WORKLOADS["x8"].replace(M=37, noise_dist=dist, noise_scale=scale, crosstalk=terms)
        u, mask, _, ins, tgs = case(w)
        ctx = gpu_context(w, ins, tgs, mask)
        ctx.sample_noise(w.seed_J, dist, scale)
        Jg = ctx.get_noise()
        Jo = noise.sample_J(w.seed_J, w.M, w.N, dist, scale, terms=terms)
        if dist == 0:
            assert np.array_equal(Jg, Jo)
        else:
            assert np.max(np.abs(Jg - Jo)) <= 1e-15 * np.max(np.abs(Jo)) * 10


def test_repeat_calls_are_bitwise_deterministic():
    w = synth.WORKLOADS["x8"].replace(M=4)
    u, mask, J, ins, tgs = case(w)
    ctx = gpu_context(w, ins, tgs, mask)
    ctx.set_controls(u)
    ctx.set_noise(J)
    a = ctx.fidelity_grad()
    b = ctx.fidelity_grad()
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_state_errors_and_recovery():
    from paper_2603_03639_gb300 import TNRCError
    w = synth.WORKLOADS["x8"].replace(M=2, K=2)
    u, mask, J, ins, tgs = case(w)
    ctx = gpu_context(w, ins, tgs, mask)
    with pytest.raises(TNRCError) as e:
        ctx.fidelity()
    assert e.value.status == -4
    with pytest.raises(TNRCError):
        ctx.set_controls(u[:1])
    ctx.set_controls(u)
    with pytest.raises(TNRCError):
        ctx.set_noise(np.full_like(J, np.nan))
    ctx.set_noise(J)
    F = ctx.fidelity()
    assert 0.0 <= F <= 1.0


@pytest.mark.parametrize("name", ["x50", "cnot50", "ghz30"])
def test_full_size_sampled_trajectories(name):
    """Full N, K, chi in the benchmark's launch configuration (the autotuned
    shape bench.py uses), reduced to a few noise samples: every overlap
    against the oracle, and the gradient of a one-trajectory ensemble."""
    from paper_2603_03639_gb300 import autotune
    w0 = synth.WORKLOADS[name]
    warps, ctas = autotune.lookup(w0.N, w0.K, w0.chi, w0.M, w0.P, w0.C, grad=True)
    w = w0.replace(M=2, P=min(2, w0.P))
    u, mask, J, ins, tgs = case(w)
    ctx = gpu_context(w, ins, tgs, mask, warps=warps, ctas_per_sm=ctas)
    ctx.set_controls(u)
    ctx.set_noise(J)
    F = ctx.fidelity()
    O = ctx.overlaps()
    pb = oracle_problem(w, u, mask, J, ins, tgs)
    for s in range(w.M):
        for p in range(w.P):
            o, _ = robust.trajectory(pb, s, p, want_grad=False)
            assert abs(O[s, p] - o) <= TOL_O
    w1 = w.replace(M=1, P=1)
    u, mask, J, ins, tgs = case(w1)
    ctx = gpu_context(w1, ins, tgs, mask, warps=warps, ctas_per_sm=ctas)
    ctx.set_controls(u)
    ctx.set_noise(J)
    F, g = ctx.fidelity_grad()
    Fo, go, _ = robust.ensemble(oracle_problem(w1, u, mask, J, ins, tgs))
    assert abs(F - Fo) <= TOL_F
    assert grad_close(g, go)


def test_full_size_operator_form_sampled_overlaps():
    """The operator form at the gate workload's full size (N=50, chi=20,
    K=100, its autotuned launch shape) on two noise samples, with an X-gate
    target near the pi pulse so that the overlaps are O(1): every overlap
    against the oracle.  (The gradient is checked at smaller sizes: the
    oracle's costate sweep over 80 x 80 operator thetas takes minutes.)"""
    from paper_2603_03639_gb300 import autotune
    w0 = synth.WORKLOADS["cnotgate50"]
    warps, ctas = autotune.lookup(w0.N, w0.K, w0.chi, w0.M, w0.P, w0.C, grad=True, operator=True)
    w = w0.replace(M=2, target="x", g_bonds="all")
    u = synth.pi_pulse_controls(w.K, w.C, w.N, w.dt, seed=7, jitter=0.05)
    u, mask, J, ins, tgs = case(w, u)
    ctx = gpu_context(w, ins, tgs, mask, warps=warps, ctas_per_sm=ctas)
    ctx.set_controls(u)
    ctx.set_noise(J)
    F = ctx.fidelity()
    O = ctx.overlaps()
    assert F > 0.1
    pb = oracle_problem(w, u, mask, J, ins, tgs)
    for s in range(w.M):
        o, _ = robust.trajectory(pb, s, 0, want_grad=False)
        assert abs(O[s, 0] - o) <= TOL_O


def test_packed_history_and_checkpoint_fallback_agree(monkeypatch):
    """The costate sweep reads the forward history packed (no recomputation)
    when it fits the CTA's region; a history cap of 0 forces every trajectory
    onto the checkpoint/recompute path.  Results must be identical."""
    w = synth.WORKLOADS["ghz30"].replace(N=12, K=5, chi=32, M=2, P=1, u_sigma=1.5, dt=0.25)
    u, mask, J, ins, tgs = case(w)
    out = {}
    for cap in ("none", "0"):
        if cap == "none":
            monkeypatch.delenv("TNRC_HISTORY_CAP", raising=False)
        else:
            monkeypatch.setenv("TNRC_HISTORY_CAP", cap)
        ctx = gpu_context(w, ins, tgs, mask)
        ctx.set_controls(u)
        ctx.set_noise(J)
        out[cap] = ctx.fidelity_grad()
        st = ctx.stats()
        assert st["restarts"] == (w.M * w.P if cap == "0" else 0)
    assert out["0"][0] == out["none"][0]
    assert np.array_equal(out["0"][1], out["none"][1])


def test_graph_replay_equals_plain_launches():
    """tnrc_evaluate_dev through captured CUDA graphs (with and without the
    gate rebuild) gives bitwise the plain launches' results."""
    import torch
    w = synth.WORKLOADS["x8"].replace(M=4, P=2)
    u, mask, J, ins, tgs = case(w)
    u2 = u + 0.01
    side = torch.cuda.Stream()
    stream = side.cuda_stream
    outs = {}
    from paper_2603_03639_gb300 import Context, TNRCError
    legacy = Context(w.N, w.K, w.dt, w.chi, w.M, w.C, ins, tgs, mask=mask)
    with pytest.raises(TNRCError):
        legacy.set_graphs(True)          # the legacy default stream cannot be captured
    legacy.close()
    torch.cuda.synchronize()
    for graphs in (False, True):
        ctx = Context(w.N, w.K, w.dt, w.chi, w.M, w.C, ins, tgs, mask=mask, stream=stream)
        ctx.set_graphs(graphs)
        ctx.set_noise(J)
        F = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.zeros(u.shape, dtype=torch.float64, device="cuda")
        res = []
        torch.cuda.synchronize()
        for uu in (u, u2, u2, u):
            ud = torch.tensor(uu, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            ctx.set_controls_dev(ud.data_ptr())
            ctx.evaluate_dev(F.data_ptr(), g.data_ptr())
            ctx.sync()
            res.append((F.item(), g.cpu().numpy().copy()))
        # same controls again without a new set: gates are current
        ctx.evaluate_dev(F.data_ptr(), g.data_ptr())
        ctx.sync()
        res.append((F.item(), g.cpu().numpy().copy()))
        ctx.close()
        outs[graphs] = res
    for (Fa, ga), (Fb, gb) in zip(outs[False], outs[True]):
        assert Fa == Fb and np.array_equal(ga, gb)
    assert outs[True][3][0] == outs[True][0][0]


def test_pooled_launch_equals_persistent_launch():
    """The pooled form (one CTA per trajectory, work regions from a device
    pool) gives bitwise the persistent form's results, with more trajectories
    than regions (so regions are handed from CTA to CTA) and with graphs."""
    import torch
    w = synth.WORKLOADS["cnot50"].replace(N=12, K=6, chi=16, M=100, P=2)   # 200 trajectories, 152 regions
    u, mask, J, ins, tgs = case(w)
    out = {}
    for pooled in (False, True):
        ctx = gpu_context(w, ins, tgs, mask, warps=4, ctas_per_sm=1)
        ctx.set_pooled(pooled)
        ctx.set_controls(u)
        ctx.set_noise(J)
        out[pooled] = ctx.fidelity_grad()
        ctx.close()
    assert out[True][0] == out[False][0]
    assert np.array_equal(out[True][1], out[False][1])
    side = torch.cuda.Stream()
    from paper_2603_03639_gb300 import Context
    ctx = Context(w.N, w.K, w.dt, w.chi, w.M, w.C, ins, tgs, mask=mask, stream=side.cuda_stream, warps=4,
                  ctas_per_sm=1)
    ctx.set_pooled(True)
    ctx.set_graphs(True)
    ctx.set_noise(J)
    ud = torch.tensor(u, dtype=torch.float64, device="cuda")
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(u.shape, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for _ in range(2):
        ctx.set_controls_dev(ud.data_ptr())
        ctx.evaluate_dev(F.data_ptr(), g.data_ptr())
        ctx.sync()
        assert F.item() == out[False][0] and np.array_equal(g.cpu().numpy(), out[False][1])
    ctx.close()


@pytest.mark.parametrize("name", ["truncated", "operator"])
def test_plain_path_equals_batched_launch(name):
    """tnrc_fidelity_grad_plain (one trajectory at a time, one launch per
    step) runs the batched kernel's device functions: bitwise the same F and
    gradient, and the oracle's within the bars."""
    if name == "truncated":
        w = synth.WORKLOADS["ghz30"].replace(N=12, K=4, chi=32, M=2, P=1, u_sigma=1.5, dt=0.25)
    else:
        w = synth.WORKLOADS["cnotgate50"].replace(N=6, K=3, chi=8, M=2)
    u, mask, J, ins, tgs = case(w)
    ctx = gpu_context(w, ins, tgs, mask)
    ctx.set_controls(u)
    ctx.set_noise(J)
    F, g = ctx.fidelity_grad()
    Fp, gp = ctx.fidelity_grad_plain()
    assert Fp == F and np.array_equal(gp, g)
    Fo, go, _ = robust.ensemble(oracle_problem(w, u, mask, J, ins, tgs))
    assert abs(Fp - Fo) <= TOL_F
    assert grad_close(gp, go)


@pytest.mark.parametrize("shape", [(8, 1), (4, 2)])
def test_svd_shape_pairs_and_one_per_warp(shape):
    """Both matrix shapes -- two small SVDs per warp on the half-warps, and one
    SVD per warp -- meet the oracle's bars, forward and costate, on a case
    whose bonds are small enough to pair and one with wider thetas."""
    for w in (synth.WORKLOADS["cnot50"].replace(N=12, K=6, chi=16, M=3, P=2),
              synth.WORKLOADS["ghz30"].replace(N=12, K=5, chi=32, M=1, P=1, u_sigma=1.5, dt=0.25)):
        u, mask, J, ins, tgs = case(w)
        Fo, go, Oo = robust.ensemble(oracle_problem(w, u, mask, J, ins, tgs))
        for pairs in (True, False):
            ctx = gpu_context(w, ins, tgs, mask, warps=shape[0], ctas_per_sm=shape[1])
            ctx.set_svd_shape(pairs)
            ctx.set_controls(u)
            ctx.set_noise(J)
            F, g = ctx.fidelity_grad()
            assert abs(F - Fo) <= TOL_F
            assert np.max(np.abs(ctx.overlaps() - Oo)) <= TOL_O
            assert grad_close(g, go)
            ctx.close()
