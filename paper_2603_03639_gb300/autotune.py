"""Launch-shape autotuner for the trajectory kernel.

The kernel runs one trajectory per CTA; within a CTA the warps share the
disjoint bonds of a TEBD layer.  The free choices are the warps per CTA (how
many bonds of a layer run at once, and how evenly a layer's bonds divide
among them), the resident CTAs per SM (how many trajectories interleave on an
SM; the register file holds 8 of this kernel's warps per SM) and the matrix
shape (two small SVDs per warp on the half-warps, or one SVD per warp).  The
tuner times each candidate on the actual problem with CUDA events around the
kernel and caches the fastest per shape bucket in a JSON file.

    python -m paper_2603_03639_gb300.autotune --workload cnot50 --out tuned.json
"""
import argparse
import json
import os
import sys

import numpy as np

CANDIDATES = [(8, 1), (6, 1), (5, 1), (4, 2), (4, 1), (3, 2), (2, 4), (8, 2), (4, 4), (6, 2), (5, 3)]
QUICK = [(8, 1), (4, 2), (3, 2), (8, 2), (4, 4)]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def shape_key(N, K, chi, M, P, C, grad=True, operator=False):
    """Shape bucket: N and C exactly; K, M*P and chi by powers of two; the
    operator form (physical dimension 4) apart."""
    b = lambda x: 1 << int(np.ceil(np.log2(max(1, x))))  # noqa: E731
    return "N%d-C%d-K%d-T%d-chi%d-%s%s" % (N, C, b(K), b(M * P), b(chi), "grad" if grad else "fid",
                                         "-op" if operator else "")


def load(path=None):
    path = path or os.environ.get("TNRC_AUTOTUNE_CACHE", DEFAULT_CACHE)
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(N, K, chi, M, P, C, grad=True, path=None, operator=False):
    """(warps_per_cta, ctas_per_sm) cached for this shape -- or for the same
    shape with the nearest ensemble-size bucket -- else (0, 0) (defaults)."""
    cache = load(path)
    key = shape_key(N, K, chi, M, P, C, grad, operator)
    e = cache.get(key)
    if e is None:
        head, tail = key.split("-T")
        rest = tail.split("-", 1)[1]
        t = int(tail.split("-", 1)[0])
        near = [(abs(np.log2(int(k.split("-T")[1].split("-")[0])) - np.log2(t)), k) for k in cache
                if k.startswith(head + "-T") and k.split("-T")[1].split("-", 1)[1] == rest]
        if near:
            e = cache[min(near)[1]]
    return (int(e["warps"]), int(e["ctas_per_sm"])) if e else (0, 0)


def lookup_pairs(N, K, chi, M, P, C, grad=True, path=None, operator=False):
    """The cached matrix shape for this problem: True = two small SVDs per warp
    on the half-warps (also the default when nothing is cached), False = one
    SVD per warp."""
    cache = load(path)
    key = shape_key(N, K, chi, M, P, C, grad, operator)
    e = cache.get(key)
    if e is None:
        w, c = lookup(N, K, chi, M, P, C, grad, path, operator)
        e = next((v for v in cache.values() if v.get("warps") == w and v.get("ctas_per_sm") == c
                  and v.get("operator", False) == operator), None)
    return bool(e.get("pairs", True)) if e else True


def tune(N, K, dt, chi, M, C, inputs, targets, u, noise, mask=None, grad=True, candidates=CANDIDATES, reps=1,
         stream=None, form=None):
    """Time every launch shape with paired SVDs, then the two fastest with one
    SVD per warp as well; returns (best (warps, ctas, pairs), {(warps, ctas,
    pairs): ms}).  form: Context keywords of the time discretisation and form
    (crosstalk, order, substeps, operator)."""
    from .tnrc import Context
    seed, dist, scale = noise
    form = form or {}
    nb = max((N - 1 + 1) // 2, 1)
    max_warps_per_sm = 8 if form.get("operator") else 16   # operators run the 255-register build only
    times = {}

    def run(w, c, pairs):
        with Context(N, K, dt, chi, M, C, inputs, targets, mask=mask, stream=stream, warps=w, ctas_per_sm=c,
                     **form) as ctx:
            ctx.set_svd_shape(pairs)
            ctx.set_controls(u)
            ctx.sample_noise(seed, dist, scale)
            (ctx.fidelity_grad if grad else ctx.fidelity)()          # warm-up
            ctx.stats()
            for _ in range(reps):
                (ctx.fidelity_grad if grad else ctx.fidelity)()
            st = ctx.stats()
            times[(w, c, pairs)] = st["traj_ms"] / max(1, st["traj_launches"])

    for w, c in candidates:
        if w * c > max_warps_per_sm or w > max(2, nb):
            continue
        run(w, c, True)
    for w, c, _ in sorted(times, key=times.get)[:2]:
        run(w, c, False)
    best = min(times, key=times.get)
    return best, times


def main():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cnot50", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--set", action="append", default=[], metavar="KEY=VALUE")
    ap.add_argument("--out", default=DEFAULT_CACHE)
    ap.add_argument("--fidelity-only", action="store_true")
    ap.add_argument("--quick", action="store_true", help="only the usual winners (QUICK)")
    args = ap.parse_args()
    w = synth.WORKLOADS[args.workload]
    for kv in args.set:
        key, val = kv.split("=", 1)
        w = w.replace(**{key: type(getattr(w, key))(val)})
    ins, tgs = w.states()
    grad = not args.fidelity_only
    best, times = tune(w.N, w.K, w.dt, w.chi, w.M, w.C, ins, tgs, w.controls(),
                       (w.seed_J, w.noise_dist, w.noise_scale), mask=w.mask(), grad=grad,
                       candidates=QUICK if args.quick else CANDIDATES,
                       form={"crosstalk": w.crosstalk, "order": w.order, "substeps": w.substeps,
                             "operator": w.operator})
    cache = load(args.out)
    key = shape_key(w.N, w.K, w.chi, w.M, w.P, w.C, grad, w.operator)
    name = lambda k: "%dx%d%s" % (k[0], k[1], "" if k[2] else "-warp")  # noqa: E731
    cache[key] = {"warps": best[0], "ctas_per_sm": best[1], "pairs": bool(best[2]), "workload": w.name,
                  "operator": bool(w.operator), "ms": {name(k): round(v, 3) for k, v in times.items()}}
    with open(args.out, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    print(json.dumps({"key": key, "best": name(best), "ms": {name(k): v for k, v in times.items()}}))


if __name__ == "__main__":
    main()
