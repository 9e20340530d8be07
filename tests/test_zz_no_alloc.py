"""tnrc_fidelity_static: the evaluation for callers that cannot call
cudaMalloc (a host runtime that owns every device allocation, or a process
that must not grow its device footprint).  It must give the same fidelity and
per-trajectory overlaps as the allocating path (tnrc_create + tnrc_fidelity),
call after call, since every call reuses the same static device array.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

import synth
from oracle import noise
from tests._util import TOL_F, TOL_O

pytestmark = pytest.mark.gpu


def _case(w):
    ins, tgs = w.states()
    u = w.controls()
    J = noise.sample_J(w.seed_J, w.M, w.N, w.noise_dist, w.noise_scale, terms=w.crosstalk)
    return ins, tgs, u, J, w.mask()


@pytest.mark.parametrize("name", ["x8", "cnot_small", "first_order", "operator", "heisenberg_crosstalk"])
def test_static_scratch_matches_allocating_path_twice(name):
    from paper_2603_03639_gb300 import Context, tnrc
    if name == "x8":
        w = synth.WORKLOADS["x8"]
    elif name == "heisenberg_crosstalk":
        w = synth.WORKLOADS["cnot50"].replace(N=8, K=6, chi=16, M=3, P=2, crosstalk=3, noise_dist=0,
                                              noise_scale=0.2)
    elif name == "first_order":
        w = synth.WORKLOADS["cnot50"].replace(N=10, K=6, chi=16, M=4, P=2, order=1, substeps=2)
    elif name == "operator":
        w = synth.WORKLOADS["cnotgate50"].replace(N=8, K=5, chi=8, M=4)
    else:
        w = synth.WORKLOADS["cnot50"].replace(N=10, K=8, chi=16, M=6, P=3)
    ins, tgs, u, J, mask = _case(w)
    with Context(w.N, w.K, w.dt, w.chi, w.M, w.C, ins, tgs, cutoff=w.sv_cutoff, mask=mask, order=w.order,
                 substeps=w.substeps, operator=w.operator, crosstalk=w.crosstalk) as ctx:
        ctx.set_controls(u)
        ctx.set_noise(J)
        F_ref, pt_ref = ctx.fidelity(per_traj=True)
    for _ in range(2):
        F, pt = tnrc.fidelity_static(w.N, w.K, w.dt, w.chi, w.C, ins, tgs, u, J, cutoff=w.sv_cutoff, mask=mask,
                                     per_traj=True, order=w.order, substeps=w.substeps, operator=w.operator,
                                     crosstalk=w.crosstalk)
        assert abs(F - F_ref) <= TOL_F
        assert np.max(np.abs(pt - pt_ref)) <= TOL_O


def test_static_calls_leave_device_memory_unchanged():
    """After one warm-up call (which places the static array on the device
    under lazy module loading), further calls take no device memory: the
    driver's free-memory figure is the same before and after them."""
    import torch
    from paper_2603_03639_gb300 import tnrc
    w = synth.WORKLOADS["cnot50"].replace(N=10, K=8, chi=16, M=6, P=3)
    ins, tgs, u, J, mask = _case(w)
    F0 = tnrc.fidelity_static(w.N, w.K, w.dt, w.chi, w.C, ins, tgs, u, J, mask=mask)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        F = tnrc.fidelity_static(w.N, w.K, w.dt, w.chi, w.C, ins, tgs, u, J, mask=mask)
        assert F == F0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_scratch_rejects_oversize_problems():
    from paper_2603_03639_gb300 import tnrc
    w = synth.WORKLOADS["cnot50"].replace(M=64)
    ins, tgs, u, J, mask = _case(w)
    with pytest.raises(tnrc.TNRCError) as e:
        tnrc.fidelity_static(w.N, w.K, w.dt, w.chi, w.C, ins, tgs, u, J, mask=mask)
    assert e.value.status == -7
    # the same validation rules as tnrc_create: a non-finite fixed coupling is invalid
    w = synth.WORKLOADS["x8"].replace(M=2)
    ins, tgs, u, J, mask = _case(w)
    gfix = np.zeros((w.K, w.N - 1))
    gfix[1, 2] = np.inf
    with pytest.raises(tnrc.TNRCError) as e:
        tnrc.fidelity_static(w.N, w.K, w.dt, w.chi, w.C, ins, tgs, u, J, mask=mask, g_fixed=gfix)
    assert e.value.status == -1
