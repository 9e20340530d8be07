"""Shared helpers of the test suite: build a GPU context and the oracle
problem from the same seeded inputs."""
import numpy as np

import synth
from oracle import noise, robust

TOL_F = 1e-10          # |F_gpu - F_oracle|
TOL_G_REL = 1e-8       # ||g_gpu - g_oracle|| <= TOL_G_REL ||g_oracle||
TOL_O = 1e-10          # per-trajectory overlap


def oracle_problem(w, u, mask, J, inputs, targets, g_fixed=None):
    return robust.Problem(N=w.N, K=w.K, dt=w.dt, C=w.C, chi=w.chi, u=u, mask=mask, J=J,
                          inputs=[m.sites for m in inputs], targets=[m.sites for m in targets],
                          g_fixed=g_fixed, eps=w.sv_cutoff, order=w.order, substeps=w.substeps,
                          operator=w.operator)


def gpu_context(w, inputs, targets, mask, g_fixed=None, checkpoint_every=0, warps=0, ctas_per_sm=0):
    from paper_2603_03639_gb300 import Context
    return Context(w.N, w.K, w.dt, w.chi, w.M, w.C, inputs, targets, cutoff=w.sv_cutoff, mask=mask,
                   g_fixed=g_fixed, checkpoint_every=checkpoint_every, crosstalk=w.crosstalk, warps=warps,
                   ctas_per_sm=ctas_per_sm, order=w.order, substeps=w.substeps, operator=w.operator)


def case(w, u=None):
    """(u, mask, J, inputs, targets) for workload w with oracle-drawn noise."""
    ins, tgs = w.states()
    u = w.controls() if u is None else u
    J = noise.sample_J(w.seed_J, w.M, w.N, w.noise_dist, w.noise_scale, terms=w.crosstalk)
    return u, w.mask(), J, ins, tgs


def grad_close(g, gref):
    nref = np.linalg.norm(gref)
    return np.linalg.norm(g - gref) <= TOL_G_REL * nref and np.max(np.abs(g - gref)) <= TOL_G_REL * np.max(np.abs(gref))
