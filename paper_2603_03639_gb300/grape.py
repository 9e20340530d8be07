"""Robust GRAPE outer loop (Sec. II): minimise the ensemble-averaged
infidelity 1 - F(u) with L-BFGS, F and dF/du from the tnrc costate kernel.

  * two-stage ensemble: optimise on M samples, then estimate the infidelity
    on a larger, independent ensemble of 5M samples;
  * warm starts over the noise strength: the solution at dJ seeds the run at
    dJ + step (the paper raises dJ in 1 % steps of the main energy scale).
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
    from scipy.optimize import minimize
    seed, dist, scale = noise
    ctx.sample_noise(seed, dist, scale)
    shape = u0.shape
    free = np.ones(shape, dtype=bool) if mask is None else np.broadcast_to(mask.astype(bool)[None], shape)
    base = u0.copy()
    hist, nev = [], [0]

    def fun(x):
        u = base.copy()
        u[free] = x
        ctx.set_controls(u)
        F, g = ctx.fidelity_grad()
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
