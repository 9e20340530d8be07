"""Benchmark: fwd+adjoint MPS slice-steps/s of the tensor-network robust
GRAPE hot path (ensemble fidelity + costate gradient) on the parallel-CNOT
workload N = 50, chi_max = 64, K = 100, M = 256, P = 8, C = 3.

One step = one full evaluation through the C ABI on device-resident inputs:
noise draw (device SplitMix64), layer-gate build, forward TEBD of all M*P
trajectories (their layer history kept packed), overlaps, costate sweep with
environments and gradient, and the fixed-order ensemble reduction.
value = M*P*K slice-steps per second (whole job; N GPUs each evaluate their
own shard of noise samples).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

--impl reference times the CPU oracle (NumPy/LAPACK) on the host cores on a
bounded sample of the same workload.  --plain compares one CTA (one
trajectory at a time) with the persistent launch on a sample; --serving runs
the serving rate sweep; --workload picks another shape (x8, x50, ghz30, the
near-solution cnot50near, echo14 whose bonds reach the cap chi = 64, the
operator-form cnotgate50); --set KEY=VALUE overrides a field (profiling cases).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

DEFAULT_WORKLOAD = "cnot50"
METRIC = "fwd+adjoint MPS slice-steps/s (N=50,chi=64,M=256)"
UNIT = "slice-steps/s"
SM_COUNT = 152
FP64_FMA_PER_CLK_PER_SM = 2        # GB300: 1.25 TFLOP/s FP64 nominal at 2070 MHz x 152 SMs
SM_MAX_MHZ = 2070.0
REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


def fp64_peak_tflops():
    """FP64 FMA peak derived from unit counts and the maximum SM clock."""
    return 2.0 * FP64_FMA_PER_CLK_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12


def form_kwargs(w):
    """Context keyword arguments for the workload's time discretisation and form."""
    return {"crosstalk": w.crosstalk, "order": w.order, "substeps": w.substeps, "operator": w.operator}


def workload_config(w):
    kind = {"x": "parallel X", "cnot": "parallel CNOT", "ghz": "GHZ preparation",
            "heisenberg": "Heisenberg ground state", "input": "echo back to the input"}[w.target]
    if w.operator:
        kind += " gate (MPO from the identity, |tr(U_T^dag U)/2^N|^2)"
    ctl = {"random": "controls N(0,%g^2)" % w.u_sigma,
           "near": "near-solution controls (pi pulse + N(0,0.05^2))",
           "echo": "echo controls (N(0,%g^2), then reversed and negated)" % w.u_sigma}[w.u_mode]
    cfg = {"workload": "%s: %s on N=%d, chi_max=%d, K=%d, dt=%g, C=%d, M=%d, P=%d, %s J, %s"
                       % (w.name, kind, w.N, w.chi, w.K, w.dt, w.C, w.M, w.P,
                          ("U[-%g,%g]" % (w.noise_scale, w.noise_scale)) if w.noise_dist == 0
                          else ("N(0,%g^2)" % w.noise_scale), ctl),
           "N": w.N, "chi_max": w.chi, "K": w.K, "M": w.M, "P": w.P, "C": w.C, "dt": w.dt,
           "slice_steps_per_eval": w.slice_steps}
    if w.order != 2 or w.substeps != 1 or w.crosstalk != 1 or w.operator:
        cfg.update(trotter_order=w.order, substeps=w.substeps, crosstalk_terms=w.crosstalk, operator=w.operator)
    return cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 4:
                try:
                    self.rows.append((float(parts[0]), float(parts[1]), float(parts[2]), int(parts[3], 16)))
                except ValueError:
                    pass

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        busy = [r for r in self.rows if not (r[3] & 0x1)] or self.rows
        reasons = set()
        for r in busy:
            for bit, name in REASON_BITS.items():
                if r[3] & bit and bit != 0x1:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in busy), "sm_max_mhz": max(r[1] for r in busy),
                "power_w_max": max(r[2] for r in busy), "samples": len(busy), "reasons": sorted(reasons)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------
# CPU oracle leg
# --------------------------------------------------------------------------

def oracle_sample(w, n_traj, K_s, workers):
    """Time the oracle (fwd + costate gradient) on n_traj trajectories of the
    first K_s slices of workload w, one trajectory per spawn worker."""
    from oracle import noise, robust, runner
    ws = w.replace(K=K_s)
    prob = synth.make_problem(ws)
    J = noise.sample_J(w.seed_J, n_traj, w.N, w.noise_dist, w.noise_scale, terms=w.crosstalk)
    pb = robust.from_workload(prob, J)
    pairs = [(s, 0) for s in range(n_traj)]
    _, secs, used = runner.run(pb, pairs, want_grad=True, workers=workers)
    return n_traj * K_s, secs, used


def cpu_baseline(w, budget_steps=1):
    workers = os.cpu_count() or 1
    units, secs, used = oracle_sample(w, workers, w.K, workers)
    u1, s1, _ = oracle_sample(w, 1, w.K, 1)
    return {"value": units / secs, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": "%d trajectories (noise samples 0..%d, input 0) x all %d slices, fwd+adjoint, "
                      "one per spawn worker, OMP/BLAS 1 thread each: %.1f s" % (used, used - 1, w.K, secs),
            "single_core": {"value": u1 / s1, "unit": UNIT, "cores": 1,
                            "sample": "1 trajectory (noise sample 0, input 0) x all %d slices, fwd+adjoint, "
                                      "one spawn worker, BLAS 1 thread: %.1f s" % (w.K, s1)}}


def reference_arm(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    workers = os.cpu_count() or 1
    total = args.steps + args.warmup
    K_s = w.K if total <= 6 else max(5, (6 * w.K) // total)
    for _ in range(args.warmup):
        oracle_sample(w, workers, K_s, workers)
    times, units = [], 0
    for _ in range(args.steps):
        u, secs, used = oracle_sample(w, workers, K_s, workers)
        times.append(secs)
        units += u
    tot = sum(times)
    value = units / tot
    sample = ("%d trajectories x first %d of %d slices per step, fwd+adjoint, one per spawn worker "
              "(OMP/BLAS 1 thread each)" % (workers, K_s, w.K))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU leg
# --------------------------------------------------------------------------

KERNEL_SOURCES = ("svd_warp.cuh", "tnrc_device.cuh", "traj.cu")


def recorded_counters(workload):
    """ncu counters of the trajectory kernel recorded for this workload in
    profiles/traj_kernel_<workload>_counters.txt -- DRAM bytes per slice-step
    and executed FP64 flops per algorithmic flop, both from one capture of a
    cut of the workload -- or None when there is no record or the kernel
    sources have changed since it was taken (the record holds their SHA-256)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traj_kernel_%s_counters.txt" % workload)
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        key, sep, val = line.partition(":")
        if sep and key.strip() and " " not in key.strip():
            rec[key.strip()] = val.strip()
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2603_03639_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    if rec.get("workload") != workload or rec.get("kernel_sources_sha256") != h.hexdigest():
        return None
    try:
        return {"bytes_per_slice_step": float(rec["dram_bytes_per_slice_step"]),
                "executed_per_alg": float(rec["executed_fp64_flops_per_alg_flop"]),
                "fp64_pipe_pct": float(rec["fp64_pipe_active_pct"])}
    except (KeyError, ValueError):
        return None


def gpu_arm(args, w):
    import torch
    import torch.distributed as dist

    from paper_2603_03639_gb300 import Context

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ins, tgs = w.states()
    mask = w.mask()
    u = w.controls()
    from paper_2603_03639_gb300 import autotune
    tuned = autotune.lookup(w.N, w.K, w.chi, w.M, w.P, w.C, grad=True, operator=w.operator)
    ctx = Context(w.N, w.K, w.dt, w.chi, w.M, w.C, ins, tgs, cutoff=w.sv_cutoff, mask=mask,
                  stream=stream.cuda_stream, warps=tuned[0], ctas_per_sm=tuned[1], **form_kwargs(w))
    pairs = autotune.lookup_pairs(w.N, w.K, w.chi, w.M, w.P, w.C, grad=True, operator=w.operator)
    ctx.set_svd_shape(pairs)
    u_dev = torch.tensor(u, dtype=torch.float64, device=dev)
    F_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    g_dev = torch.zeros(u.shape, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    from paper_2603_03639_gb300.ensemble import allreduce_mean, shard_seed

    def step_seed(i):
        # step i draws a fresh global ensemble of world*M samples; this rank
        # evaluates its slice of it
        return shard_seed(w.seed_J + 7919 * i, rank, w.M, w.N, w.noise_dist, terms=w.crosstalk)

    def step(i):
        ctx.set_controls_dev(u_dev.data_ptr())
        ctx.sample_noise(step_seed(i), w.noise_dist, w.noise_scale)
        ctx.evaluate_dev(F_dev.data_ptr(), g_dev.data_ptr())
        if world > 1:
            allreduce_mean(F_dev, g_dev)           # the ensemble mean over all ranks

    for i in range(args.warmup):
        step(i)
    ctx.sync()
    ctx.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    per_step, alg, traj_ms, launches = [], 0.0, 0.0, 0
    hist = np.zeros(w.chi + 1, dtype=np.int64)
    disc, sweeps, updates, maxb, capcuts, mingap = 0.0, 0, 0, 0, 0, None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()                      # evict L2 (129 MB) between timed steps
            ev[i][0].record(stream)
            step(args.warmup + i)
            ev[i][1].record(stream)
            ev[i][1].synchronize()
            per_step.append(ev[i][0].elapsed_time(ev[i][1]))
            st = ctx.stats()
            ctx.sync()
            alg += st["alg_flops"]
            traj_ms += st["traj_ms"]
            launches += st["traj_launches"]
            hist += np.asarray(st["bond_hist"], dtype=np.int64)
            disc += st["discarded_weight"]
            sweeps += st["jacobi_sweeps"]
            updates += st["updates"]
            maxb = max(maxb, st["max_bond"])
            capcuts += st["cap_truncations"]
            if st["min_trunc_gap"] >= 0.0:
                mingap = st["min_trunc_gap"] if mingap is None else min(mingap, st["min_trunc_gap"])
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = sum(per_step)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    value = world * w.slice_steps / (ms_per_step / 1000.0)

    # end to end through the host-buffer C ABI: controls in, F and gradient out
    u_pin = torch.tensor(u, dtype=torch.float64).pin_memory().numpy()
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        ctx.set_controls(u_pin)
        ctx.sample_noise(step_seed(args.warmup + args.steps + i), w.noise_dist, w.noise_scale)
        F_h, g_h = ctx.fidelity_grad()
        if world > 1:
            Ft, gt = torch.tensor([F_h], device=dev), torch.tensor(g_h, device=dev)
            allreduce_mean(Ft, gt)
            F_h, g_h = Ft.item(), gt.cpu().numpy()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    KCN = w.K * w.C * w.N

    peak = fp64_peak_tflops()
    from paper_2603_03639_gb300.tnrc import measure_fp64_peak
    probe = torch.empty(4 * 256 * torch.cuda.get_device_properties(dev).multi_processor_count,
                        dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    measured_peak = measure_fp64_peak(probe.data_ptr(), probe.numel() * 8) / 1e3
    from paper_2603_03639_gb300.tnrc import measure_dmma_peak
    measured_dmma = measure_dmma_peak(probe.data_ptr(), probe.numel() * 8) / 1e3
    achieved = (alg / launches) / (traj_ms / launches / 1000.0) / 1e12 if launches else None
    rec = recorded_counters(w.name)
    traffic = int(rec["bytes_per_slice_step"] * w.slice_steps) if rec else None
    # executed FP64 work: the recorded ratio of executed (2 DFMA + DADD + DMUL,
    # thread level) to algorithmic flops applied to this launch's algorithmic rate
    exec_tf = achieved * rec["executed_per_alg"] if (rec and achieved) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(w), parallelism="ensemble-sharded x%d (noise samples per GPU)" % world,
                       l2="flushed between timed steps (512 MB write, outside the per-step events)"),
        "e2e": {"value": world * w.slice_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": KCN * 8,
                "d2h_bytes_per_step": 8 + KCN * 8},
        # per step: noise_kernel, layer_gate_kernel, traj_kernel, reduce_fidelity_kernel,
        # reduce_grad_kernel (the launch list under profiles/ shows the same five)
        "gpu_launches": 5 * args.steps,
        "launch_shape": {"warps_per_cta": tuned[0] or "default", "ctas_per_sm": tuned[1] or 1,
                         "svd": "two per warp (half-warps)" if pairs else "one per warp",
                         "source": "autotune cache" if tuned[0] else "default"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "frac_executed": (exec_tf / peak) if exec_tf else None,
                     "frac_note": ("frac divides the nominal algorithmic count (the thin-SVD formula on the "
                                   "full theta, contractions, environments) by the kernel time; frac_executed "
                                   "divides the FP64 work the kernel executed (ncu)"
                                   + ("; a nominal frac above about 1.2 reflects the count, not the pipe"
                                      if achieved and achieved / peak > 1.2 else "")),
                     "executed_tflops": exec_tf,
                     "counters_source": ("ncu counters of a cut of this workload, per slice-step "
                                         "(profiles/traj_kernel_%s_counters.txt)" % w.name)
                     if rec else "no ncu record for these kernel sources",
                     "kernel": "tnrc::traj_kernel",
                     "peak_source": "derived FP64 FMA peak: 2 DFMA/clk/SM x 152 SMs x 2070 MHz",
                     "measured_fp64_fma_peak": measured_peak,
                     "measured_fp64_dmma_peak": measured_dmma,
                     "frac_of_measured": (achieved / measured_peak) if achieved and measured_peak else None},
        "clocks": clk.summary(),
        "workload_stats": {"alg_flops_per_step": alg / args.steps, "traj_kernel_ms_per_step": traj_ms / args.steps,
                           "max_bond": maxb, "bond_hist": hist.tolist(), "discarded_weight": disc / args.steps,
                           "jacobi_sweeps_per_update": sweeps / max(1, updates),
                           "updates_per_step": updates / args.steps,
                           # cuts the cap chi_max decided (more values above the cutoff than it
                           # keeps) and their smallest (sigma_k - sigma_k+1) / sigma_1; below
                           # 1e-10 a cut is a tie
                           "cap_truncations_per_step": capcuts / args.steps, "min_trunc_gap": mingap,
                           "tie_at_cut": bool(mingap is not None and mingap < 1e-10)},
    }
    if rank == 0 and world == 1 and not args.no_serving:
        line["serving"] = serving_block(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# serving leg
# --------------------------------------------------------------------------

def serving_problems(mix="bench", seed=41):
    """Eight resident problems ("optimisers") drawn like the mixed serving
    workload: N in {8, 20, 30, 50} (two of each), chi in {16, 32, 64}, K and M
    log-uniform.  N=8: parallel X (P=4); N=20: the Heisenberg ground state
    from |0..0> at the paper's D_max = 20 (chi 20); N=30: GHZ; N=50: parallel
    X or CNOT by the problem's parity (P=2).
      mix "bench":   K in [20, 50], M in [4, 32] (a sweep ends in seconds);
      mix "config5": K in [20, 200], M in [16, 512] (the full ranges)."""
    lo_k, hi_k, lo_m, hi_m = (20, 50, 4, 32) if mix == "bench" else (20, 200, 16, 512)
    rng = np.random.default_rng(seed)
    probs = []
    heis = {}
    for j in range(8):
        N = [8, 20, 30, 50][j % 4]
        chi = int(rng.choice([16, 32, 64]))
        K = int(round(np.exp(rng.uniform(np.log(lo_k), np.log(hi_k)))))
        M = int(round(np.exp(rng.uniform(np.log(lo_m), np.log(hi_m)))))
        if N == 8:
            w = synth.WORKLOADS["x8"].replace(chi=min(chi, 16), K=K, M=M)
        elif N == 20:
            w = synth.Workload("heis20", N=20, chi=20, K=K, dt=0.05, C=3, M=M, P=1, noise_dist=0,
                               noise_scale=0.05, seed_u=100 + j, seed_J=200 + j, seed_in=300 + j,
                               target="heisenberg", g_bonds="all")
        elif N == 30:
            w = synth.WORKLOADS["ghz30"].replace(chi=chi, K=K, M=M)
        else:
            base = "cnot50" if (j // 4) % 2 else "x50"
            w = synth.WORKLOADS[base].replace(chi=chi, K=K, M=M, P=2)
        if w.target == "heisenberg":
            if w.chi not in heis:
                heis[w.chi] = w.states()
            ins, tgs = heis[w.chi]
        else:
            ins, tgs = w.states()
        probs.append((("p%d" % j), w, ins, tgs))
    return probs


def serving_requests(probs, rate, n_req, seed):
    """A Poisson request stream over the resident problems: (arrival times,
    requests), controls N(0, 0.5^2), own noise seed, half with gradient."""
    from paper_2603_03639_gb300.serving import Request
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    reqs = []
    for _ in range(n_req):
        key, w, ins, tgs = probs[int(rng.integers(len(probs)))]
        reqs.append(Request(key=key, N=w.N, K=w.K, dt=w.dt, chi=w.chi, M=w.M, C=w.C, inputs=ins, targets=tgs,
                            controls=rng.normal(0, 0.5, size=(w.K, w.C, w.N)),
                            noise_seed=int(rng.integers(1 << 40)), noise_dist=w.noise_dist,
                            noise_scale=w.noise_scale, want_grad=bool(rng.integers(2)), mask=w.mask()))
    return arrivals, reqs


def _summary(reqs, rate, extra=None):
    from paper_2603_03639_gb300.serving import latency_stats
    st = latency_stats(reqs)
    st["offered_rps"] = rate
    # per size class (chain length): p50/p99 latency of that class's requests
    st["by_N"] = {}
    for n in sorted({r.N for r in reqs}):
        sub = latency_stats([r for r in reqs if r.N == n])
        st["by_N"][str(n)] = {k: sub[k] for k in ("n", "p50_s", "p99_s") if k in sub}
    if extra:
        st.update(extra)
    return st


def served_run(probs, arrivals, reqs, max_inflight=8):
    """The continuous-batching server (pooled launches, priority streams)."""
    from paper_2603_03639_gb300.serving import Request, Server
    srv = Server(max_inflight=max_inflight)
    # make every problem resident first, two copies each (context creation is
    # not request latency, and two requests of one problem can then be in
    # flight at once), and let the server measure their sizes
    for key, w, ins, tgs in probs:
        for _ in range(2):
            for _ in range(2):
                srv.submit(Request(key=key, N=w.N, K=w.K, dt=w.dt, chi=w.chi, M=w.M, C=w.C, inputs=ins,
                                   targets=tgs, controls=np.zeros((w.K, w.C, w.N)), noise_seed=1,
                                   noise_dist=w.noise_dist, noise_scale=w.noise_scale, want_grad=True,
                                   mask=w.mask()))
            srv.drain()
    t0 = time.perf_counter()
    for r, t in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        srv.submit(r)
    srv.drain()
    peak = srv.peak_inflight
    made = len(srv.slots)
    srv.close()
    return {"peak_inflight": peak, "high_priority": sum(1 for r in reqs if r.priority == "high"),
            "resident_contexts": made}


def plain_run(probs, arrivals, reqs):
    """Plain sequential GPU calls: the same resident contexts (persistent
    launch, CUDA graph), one request at a time in arrival order."""
    import torch

    from paper_2603_03639_gb300 import Context
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    ctxs = {}
    F = torch.zeros(1, dtype=torch.float64, device=dev)
    for key, w, ins, tgs in probs:
        ctx = Context(w.N, w.K, w.dt, w.chi, w.M, w.C, ins, tgs, cutoff=w.sv_cutoff, mask=w.mask(),
                      stream=stream.cuda_stream, **form_kwargs(w))
        ctx.set_graphs(True)
        g = torch.zeros((w.K, w.C, w.N), dtype=torch.float64, device=dev)
        for grad in (True, False):           # capture both graphs before the clock starts
            ctx.set_controls(np.zeros((w.K, w.C, w.N)))
            ctx.sample_noise(1, w.noise_dist, w.noise_scale)
            ctx.evaluate_dev(F.data_ptr(), g.data_ptr() if grad else 0)
            ctx.sync()
        ctxs[key] = (ctx, g)
    t0 = time.perf_counter()
    for r, t in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        r.arrival = t0 + t
        ctx, g = ctxs[r.key]
        r.start = time.perf_counter()
        ctx.set_controls(r.controls)
        ctx.sample_noise(r.noise_seed, r.noise_dist, r.noise_scale)
        ctx.evaluate_dev(F.data_ptr(), g.data_ptr() if r.want_grad else 0)
        ctx.sync()
        r.F = float(F.item())
        r.grad = g.cpu().numpy().copy() if r.want_grad else None
        r.finish = time.perf_counter()
    for ctx, _ in ctxs.values():
        ctx.close()
    return {}


def serving_compare(probs, rate, n_req, seed):
    """Served vs plain on one request stream; every result must agree bitwise."""
    import copy
    arrivals, reqs = serving_requests(probs, rate, n_req, seed)
    reqs_p = [copy.copy(r) for r in reqs]
    ex = served_run(probs, arrivals, reqs)
    served = _summary(reqs, rate, ex)
    plain = _summary(reqs_p, rate, plain_run(probs, arrivals, reqs_p))
    same = all(a.error is None and b.error is None and a.F == b.F
               and (a.grad is None or np.array_equal(a.grad, b.grad)) for a, b in zip(reqs, reqs_p))
    return {"offered_rps": rate, "requests": n_req, "served": served, "plain": plain, "results_identical": same}


def serving_block(args):
    """The served half of the metric on the bench mix, for the headline line."""
    probs = serving_problems("bench")
    row = serving_compare(probs, args.serve_rate, args.serve_requests, 4242)
    row["mix"] = [{"key": k, "N": w.N, "chi": w.chi, "K": w.K, "M": w.M, "P": w.P, "target": w.target}
                  for k, w, _, _ in probs]
    row["what"] = ("Poisson requests over 8 resident problems (bench mix: N in {8,20,30,50}, K in [20,50], "
                   "M in [4,32]); served = continuous batching (pooled launches, priority streams); plain = the "
                   "same requests as sequential GPU calls in arrival order")
    return row


def serving_arm(args):
    probs = serving_problems(args.mix)
    rates = [float(x) for x in args.rates.split(",")]
    rows = []
    for rate in rates:
        row = serving_compare(probs, rate, args.requests, 1000 + int(rate * 10))
        print("at %g req/s: %s" % (rate, json.dumps(row)), file=sys.stderr, flush=True)
        rows.append(row)
    line = {"metric": "served p50/p99 latency and throughput vs plain sequential GPU calls",
            "unit": "s, req/s", "mix_name": args.mix,
            "mix": [{"key": k, "N": w.N, "chi": w.chi, "K": w.K, "M": w.M, "P": w.P,
                     "target": w.target} for k, w, _, _ in probs],
            "requests_per_rate": args.requests, "max_inflight": 8, "sweep": rows, "data": "synthetic"}
    print(json.dumps(line), flush=True)


def plain_arm(args, w):
    """Plain vs batched on the same sample of the workload (`--plain-samples`
    noise samples, all P inputs and K slices), both through the C ABI on one
    context, each timed over `--steps` repeats after a warm-up:
      batched   the persistent launch over all SMs (the headline form);
      plain     tnrc_fidelity_grad_plain: one trajectory at a time, one launch
                per step, the layer's bonds spread over CTAs -- the whole GPU
                for one trajectory;
      one_cta   the persistent kernel with a single CTA (one trajectory at a
                time on one SM).
    Prints one JSON line; every form's F and gradient must agree bitwise."""
    import torch

    from paper_2603_03639_gb300 import Context, autotune

    ws = w.replace(M=args.plain_samples)
    ins, tgs = ws.states()
    tuned = autotune.lookup(w.N, w.K, w.chi, w.M, w.P, w.C, grad=True, operator=w.operator)
    out, ref = {}, None
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for mode in ("batched", "plain", "one_cta"):
            if mode == "one_cta":
                os.environ["TNRC_GRID"] = "1"
            try:
                ctx = Context(ws.N, ws.K, ws.dt, ws.chi, ws.M, ws.C, ins, tgs, cutoff=ws.sv_cutoff,
                              mask=ws.mask(), warps=tuned[0], ctas_per_sm=tuned[1], **form_kwargs(ws))
            finally:
                os.environ.pop("TNRC_GRID", None)
            ctx.set_svd_shape(autotune.lookup_pairs(w.N, w.K, w.chi, w.M, w.P, w.C, grad=True,
                                                    operator=w.operator))
            ctx.set_controls(ws.controls())
            ctx.sample_noise(ws.seed_J, ws.noise_dist, ws.noise_scale)
            run = ctx.fidelity_grad_plain if mode == "plain" else ctx.fidelity_grad
            run()                                  # warm-up
            torch.cuda.synchronize()
            reps = 1 if mode == "one_cta" else max(1, args.steps)
            secs = []
            for _ in range(reps):
                t0 = time.perf_counter()
                F, g = run()
                secs.append(time.perf_counter() - t0)
            sec = statistics.median(secs)
            out[mode] = {"value": ws.slice_steps / sec, "s_per_eval": sec, "repeats": reps, "F": float(F)}
            if ref is None:
                ref = (F, g)
            out[mode]["identical_to_batched"] = bool(F == ref[0] and np.array_equal(g, ref[1]))
            ctx.close()
    line = {"metric": "batched persistent launch vs plain one-trajectory-at-a-time GPU paths", "unit": UNIT,
            "workload": w.name, "sample": "M=%d noise samples x P=%d inputs x K=%d slices, fwd+adjoint"
            % (ws.M, ws.P, ws.K), "batched": out["batched"], "plain": out["plain"], "one_cta": out["one_cta"],
            "speedup_vs_plain": out["batched"]["value"] / out["plain"]["value"],
            "speedup_vs_one_cta": out["batched"]["value"] / out["one_cta"]["value"],
            "results_identical": all(v["identical_to_batched"] for v in out.values()),
            "launch_shape": {"warps_per_cta": tuned[0] or "default", "ctas_per_sm": tuned[1] or 1},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tnrc", choices=["tnrc", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", action="store_true", help="serving rate sweep (separate JSON line)")
    ap.add_argument("--mix", default="bench", choices=["bench", "config5"], help="serving problem mix")
    ap.add_argument("--rates", default="8,32")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--no-serving", action="store_true", help="leave the serving block out of the bench line")
    ap.add_argument("--serve-rate", type=float, default=8.0)
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--plain", action="store_true",
                    help="plain (one CTA) vs batched launch on a sample of the workload (separate JSON line)")
    ap.add_argument("--plain-samples", type=int, default=2)
    ap.add_argument("--set", action="append", default=[], metavar="KEY=VALUE",
                    help="override a workload field (profiling cases), e.g. --set K=10 --set M=19")
    args = ap.parse_args()
    w = synth.WORKLOADS[args.workload]
    for kv in args.set:
        key, val = kv.split("=", 1)
        cur = getattr(w, key)
        w = w.replace(**{key: type(cur)(val)})
    if args.serving:
        serving_arm(args)
    elif args.plain:
        plain_arm(args, w)
    elif args.impl == "reference":
        reference_arm(args, w)
    else:
        gpu_arm(args, w)


if __name__ == "__main__":
    main()
