"""Host logic of bench.py on the CPU: the ncu counters record is used only
while the kernel sources hash to the SHA-256 it was taken under, and only
for its own workload."""
import hashlib
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture()
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(HERE, "..", "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _tree(tmp_path, bench, workload="cnot50", sha=None, sources=("a", "b", "c")):
    csrc = tmp_path / "paper_2603_03639_gb300" / "csrc"
    csrc.mkdir(parents=True)
    h = hashlib.sha256()
    for name, text in zip(bench.KERNEL_SOURCES, sources):
        (csrc / name).write_text(text)
        h.update(text.encode())
    (tmp_path / "profiles").mkdir()
    rec = ("ncu counters\n\nworkload: %s\nkernel_sources_sha256: %s\ndram_bytes_per_slice_step: 1234.5\n"
           "executed_fp64_flops_per_alg_flop: 0.5\nfp64_pipe_active_pct: 77.0\n\n| counter | value |\n"
           % (workload, sha or h.hexdigest()))
    (tmp_path / "profiles" / "traj_kernel_cnot50_counters.txt").write_text(rec)
    bench.ROOT = str(tmp_path)
    return csrc


def test_record_used_while_sources_match(tmp_path, bench):
    _tree(tmp_path, bench)
    assert bench.recorded_counters("cnot50") == {"bytes_per_slice_step": 1234.5, "executed_per_alg": 0.5,
                                                 "fp64_pipe_pct": 77.0}


def test_record_dropped_when_a_source_changes(tmp_path, bench):
    csrc = _tree(tmp_path, bench)
    (csrc / bench.KERNEL_SOURCES[1]).write_text("b changed")
    assert bench.recorded_counters("cnot50") is None


def test_record_of_another_workload_or_missing(tmp_path, bench):
    _tree(tmp_path, bench, workload="x50")
    assert bench.recorded_counters("cnot50") is None     # the file names cnot50, its body x50
    assert bench.recorded_counters("ghz30") is None      # no file


def test_committed_records_match_the_committed_sources(bench):
    """Every record under profiles/ was taken with the kernel sources as they
    are: a kernel change needs a new capture, or the record's removal (bench.py
    then reports the executed fraction and the traffic as null)."""
    prof = os.path.join(bench.ROOT, "profiles")
    names = [f for f in os.listdir(prof) if f.startswith("traj_kernel_") and f.endswith("_counters.txt")]
    assert names
    for f in names:
        w = f[len("traj_kernel_"):-len("_counters.txt")]
        rec = bench.recorded_counters(w)
        assert rec is not None, "profiles/%s is stale for the kernel sources" % f
        assert 0.0 < rec["executed_per_alg"] < 1.0 and rec["bytes_per_slice_step"] > 0.0


def test_reference_arm_prints_the_contract_line(bench):
    """`bench.py --impl reference` (the CPU oracle timed on a bounded sample of
    the benchmark workload) prints one JSON line with the GPU arm's metric,
    unit and config, its own cpu_baseline and a zero-copy e2e block."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(HERE, "..", "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=os.path.join(HERE, ".."))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"].startswith("cnot50") and d["config"]["slice_steps_per_eval"] == 204800
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
