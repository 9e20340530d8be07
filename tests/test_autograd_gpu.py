"""torch.autograd form: backward is the costate (adjoint) kernel with
checkpoint/recompute; checked against the oracle's gradient and against
central finite differences of the GPU fidelity."""
import numpy as np
import pytest

import synth
from oracle import robust
from tests._util import TOL_F, case, grad_close, oracle_problem

pytestmark = pytest.mark.gpu


def _ctx(w, ins, tgs, mask, checkpoint_every=0):
    import torch
    from paper_2603_03639_gb300 import Context
    return Context(w.N, w.K, w.dt, w.chi, w.M, w.C, ins, tgs, cutoff=w.sv_cutoff, mask=mask,
                   checkpoint_every=checkpoint_every, stream=torch.cuda.current_stream().cuda_stream)


def test_autograd_matches_oracle_gradient():
    import torch
    from paper_2603_03639_gb300.autograd import fidelity
    w = synth.WORKLOADS["x8"].replace(M=3, P=2)
    u, mask, J, ins, tgs = case(w)
    ctx = _ctx(w, ins, tgs, mask, checkpoint_every=2)
    ctx.set_noise(J)
    ut = torch.tensor(u, dtype=torch.float64, device="cuda", requires_grad=True)
    F = fidelity(ut, ctx)
    F.backward()
    Fo, go, _ = robust.ensemble(oracle_problem(w, u, mask, J, ins, tgs))
    assert abs(F.item() - Fo) <= TOL_F
    assert grad_close(ut.grad.cpu().numpy(), go)
    # a scalar multiple of F back-propagates scaled
    ut.grad = None
    (3.0 * fidelity(ut, ctx)).backward()
    assert grad_close(ut.grad.cpu().numpy(), 3.0 * go)
    # without grad only the forward pass runs
    with torch.no_grad():
        F2 = fidelity(ut, ctx)
    assert F2.item() == F.item()


def test_autograd_central_differences_at_cnot50_scale():
    """N=50, chi=64, K=100, 3 controls per site (the costate sweep reads the
    packed forward history; the sqrt-sized checkpoint path is its fallback);
    a 2x2 ensemble keeps the 40 extra evaluations short."""
    import torch
    from paper_2603_03639_gb300.autograd import fidelity
    w = synth.WORKLOADS["cnot50"].replace(M=2, P=2)
    u, mask, J, ins, tgs = case(w)
    ctx = _ctx(w, ins, tgs, mask)
    ctx.set_noise(J)
    ut = torch.tensor(u, dtype=torch.float64, device="cuda", requires_grad=True)
    F = fidelity(ut, ctx)
    F.backward()
    g = ut.grad.cpu().numpy()
    rng = np.random.default_rng(5)
    free = np.argwhere(np.broadcast_to(mask[None], u.shape))
    picks = free[rng.choice(len(free), 20, replace=False)]
    h = 1e-6
    gmax = np.max(np.abs(g))
    with torch.no_grad():
        for idx in picks:
            idx = tuple(int(x) for x in idx)
            up = ut.detach().clone()
            um = ut.detach().clone()
            up[idx] += h
            um[idx] -= h
            fd = (fidelity(up, ctx).item() - fidelity(um, ctx).item()) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-6 * gmax, (idx, fd, g[idx])
