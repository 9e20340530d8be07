"""Process-pool map of oracle trajectories over host cores (the timed CPU
baseline).  The pool is started with the ``spawn`` method and each worker pins
its BLAS to one thread, so that the trajectories, which are independent
(Sec. II: the ensemble members are evaluated in parallel), are what runs in
parallel."""
import multiprocessing as mp
import os
import time

_PB = None


def _init(pb):
    global _PB
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    _PB = pb


def _one(args):
    from . import robust
    s, p, want_grad = args
    return s, p, robust.trajectory(_PB, s, p, want_grad)


def run(pb, pairs, want_grad=True, workers=None):
    """Evaluate ``pairs`` [(s, p)] on ``workers`` processes.  Returns
    (results {(s, p): (O, dO)}, seconds, workers)."""
    workers = workers or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers, initializer=_init, initargs=(pb,)) as pool:
        t0 = time.perf_counter()
        res = pool.map(_one, [(s, p, want_grad) for s, p in pairs], chunksize=1)
        dt = time.perf_counter() - t0
    return {(s, p): (o, d) for s, p, (o, d) in res}, dt, workers
