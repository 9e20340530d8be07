"""Robust GRAPE outer loop (Sec. II): minimise the ensemble-averaged
infidelity 1 - F(u) with L-BFGS, F and dF/du from the tnrc costate kernel.

  * two-stage ensemble: optimise on M samples, then estimate the infidelity
    on a larger, independent ensemble of 5M samples;
  * warm starts over the noise strength: the solution at dJ seeds the run at
    dJ + step (the paper raises dJ in 1 % steps of the main energy scale);
  * warm starts over the chain length: the solution for n - p sites seeds
    the run for n sites (Sec. II: the solution of size n - 1 is the initial
    guess for size n; p = 2 keeps whole CNOT pairs), the new sites taking the
    controls of the sites p places to their left;
  * evaluations either on a context the optimiser owns or as requests to a
    serving loop (``ServedObjective``), so that many optimisers share one GPU.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np

from .tnrc import Context


@dataclasses.dataclass
class Result:
    u: np.ndarray
    infidelity: float            # on the optimisation ensemble
    validation: Optional[float]  # on the 5M validation ensemble
    iterations: int
    evaluations: int
    history: List[float]


def optimise(ctx: Context, u0: np.ndarray, noise: tuple, mask: Optional[np.ndarray] = None, maxiter: int = 100,
             gtol: float = 1e-10, callback: Optional[Callable] = None) -> Result:
    """L-BFGS on 1 - F over the context's ensemble; noise = (seed, dist, scale)
    is drawn once on the device and held fixed during the run.  Masked control
    slots stay at their initial values."""
    seed, dist, scale = noise
    ctx.sample_noise(seed, dist, scale)

    def fg(u):
        ctx.set_controls(u)
        return ctx.fidelity_grad()

    return optimise_fn(fg, u0, mask=mask, maxiter=maxiter, gtol=gtol, callback=callback)


def optimise_fn(fg: Callable, u0: np.ndarray, mask: Optional[np.ndarray] = None, maxiter: int = 100,
                gtol: float = 1e-10, callback: Optional[Callable] = None) -> Result:
    """L-BFGS on 1 - F with F, dF/du = fg(u) from any evaluator (a context, a
    serving loop).  Masked control slots stay at their initial values."""
    from scipy.optimize import minimize
    shape = u0.shape
    free = np.ones(shape, dtype=bool) if mask is None else np.broadcast_to(mask.astype(bool)[None], shape)
    base = u0.copy()
    hist, nev = [], [0]

    def fun(x):
        u = base.copy()
        u[free] = x
        F, g = fg(u)
        nev[0] += 1
        hist.append(1.0 - F)
        if callback:
            callback(1.0 - F)
        return 1.0 - F, -g[free]

    res = minimize(fun, base[free], jac=True, method="L-BFGS-B",
                   options={"maxiter": maxiter, "gtol": gtol, "ftol": 1e-15})
    u = base.copy()
    u[free] = res.x
    return Result(u=u, infidelity=float(res.fun), validation=None, iterations=int(res.nit), evaluations=nev[0],
                  history=hist)


def validate(make_context: Callable[[int], Context], u: np.ndarray, M: int, noise: tuple) -> float:
    """Infidelity of controls u on an independent ensemble of 5M samples
    (the second stage of the paper's two-stage strategy)."""
    seed, dist, scale = noise
    with make_context(5 * M) as ctx:
        ctx.set_controls(u)
        ctx.sample_noise(seed, dist, scale)
        return 1.0 - ctx.fidelity()


def robust_ramp(make_context: Callable[[int], Context], u0: np.ndarray, M: int, dJ_final: float, step: float,
                dist: int = 0, seed: int = 1, mask=None, maxiter: int = 100) -> List[Result]:
    """Warm-started robust optimisation at dJ = step, 2 step, ..., dJ_final:
    each run starts from the previous solution.  Returns one Result per dJ,
    validated on 5M fresh samples."""
    out, u = [], u0.copy()
    n = max(1, int(round(dJ_final / step)))
    for j in range(1, n + 1):
        dJ = min(dJ_final, j * step)
        with make_context(M) as ctx:
            r = optimise(ctx, u, (seed + j, dist, dJ), mask=mask, maxiter=maxiter)
        r.validation = validate(make_context, r.u, M, (10_000 + seed + j, dist, dJ))
        out.append(r)
        u = r.u
    return out


def extend_controls(u: np.ndarray, n_new: int, period: int = 1) -> np.ndarray:
    """Controls u[K][C][n] of a shorter chain extended to n_new sites: every
    new site i takes the controls of site i - period (period 2 copies whole
    pairs, as the parallel CNOT needs), and for C = 3 the g slot of the old
    last site -- which had no bond -- takes the coupling of the bond period
    places to its left.  This is the initial guess of the warm start over the
    chain length (Sec. II)."""
    K, C, n = u.shape
    if n_new < n or period < 1 or period > n:
        raise ValueError("extend_controls: need n <= n_new and 1 <= period <= n")
    out = np.zeros((K, C, n_new), dtype=np.float64)
    out[:, :, :n] = u
    if C == 3 and n_new > n:
        out[:, 2, n - 1] = out[:, 2, n - 1 - period] if n - 1 - period >= 0 else 0.0
    for i in range(n, n_new):
        out[:, :, i] = out[:, :, i - period]
    if C == 3:
        out[:, 2, n_new - 1] = 0.0
    return out


def chain_ramp(make_context: Callable[[int, int], Context], u0: np.ndarray, sizes: List[int],
               M_of: Callable[[int], int], noise: tuple, period: int = 1, mask_of: Optional[Callable] = None,
               maxiter: int = 100) -> List[Result]:
    """Warm-started robust optimisation over chain lengths sizes[0] < sizes[1]
    < ...: the solution for each size, extended by ``extend_controls``, seeds
    the next (Sec. II).  make_context(n, M) builds the problem for n sites and
    M samples; M_of(n) is the optimisation ensemble (the paper's 6(n - 1));
    noise = (seed, dist, scale).  Returns one Result per size, validated on
    5 M_of(n) fresh samples."""
    seed, dist, scale = noise
    out, u = [], u0.copy()
    for j, n in enumerate(sizes):
        if u.shape[2] != n:
            u = extend_controls(u, n, period)
        mask = mask_of(n) if mask_of else None
        with make_context(n, M_of(n)) as ctx:
            r = optimise(ctx, u, (seed + j, dist, scale), mask=mask, maxiter=maxiter)
        r.validation = validate(lambda M, n=n: make_context(n, M), r.u, M_of(n), (20_000 + seed + j, dist, scale))
        out.append(r)
        u = r.u
    return out


class ServedObjective:
    """F and dF/du of one problem as requests to a ``serving.Server``: the
    optimiser's evaluations become serving traffic, sharing the GPU with every
    other client of the server.  ``template`` is a ``serving.Request`` holding
    the problem (key, shapes, inputs/targets, noise); each call submits a copy
    with the given controls and waits for it."""

    def __init__(self, server, template):
        self.server = server
        self.template = template
        self.requests = 0

    def __call__(self, u):
        import copy
        req = copy.copy(self.template)
        req.controls = np.ascontiguousarray(u, dtype=np.float64)
        req.want_grad = True
        req.F = req.grad = req.error = None
        self.server.wait(self.server.submit(req))
        self.requests += 1
        if req.error:
            raise RuntimeError(req.error)
        return req.F, req.grad
