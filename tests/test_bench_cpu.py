"""bench.py's reference arm on the CPU (the oracle on a tiny batch): one JSON
line with the contract's keys, the reference arm's own cpu_baseline and a
zero-byte e2e; a second rank prints nothing."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=600, env=e)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]


@pytest.mark.parametrize("workload", ["lognormal_batch", "uniform_pairs"])
def test_reference_line(workload):
    lines = run(["--impl", "reference", "--workload", workload, "--pairs", "200",
                 "--steps", "2", "--warmup", "1", "--cpu-seconds", "1"])
    assert len(lines) == 1
    j = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in j, k
    assert j["impl"] == "reference" and j["unit"] == "GCUPS" and j["value"] > 0
    assert j["steps"] == 2 and j["warmup"] == 1 and j["higher_is_better"] is True
    assert j["config"]["workload"] == workload and "l2" in j["config"]
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["cores"] >= 1
    assert j["e2e"] == {"value": j["value"], "unit": "GCUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_other_rank_is_silent():
    lines = run(["--impl", "reference", "--pairs", "50", "--steps", "1", "--warmup", "0",
                 "--cpu-seconds", "1"], env={"RANK": "1", "WORLD_SIZE": "2"})
    assert lines == []


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_profiled_kernel_sources_match_the_capture():
    """The traffic and mixed ceiling in the bench line come from one ncu
    capture of the packed level-2 kernel; they are reported only while its
    sources hash to the captured ones, and these sources are those."""
    b = _bench_module()
    assert b._profile_current(b.PROFILED["level"])
    assert not b._profile_current(b.PROFILED["level"] + 1)
    # traffic scales with the extensions a launch starts
    t = b.profiled_traffic(b.PROFILED["level"], 2 * b.PROFILED["items"])
    assert t == pytest.approx(2 * b.PROFILED["bytes"])


def test_mixed_ceiling_is_the_slowest_pipe():
    """min(alu / (1 - f), fma / f, issue): a stream with a share f of its
    instructions on the FMA pipe, the rest on the ALU pipe, one issue port."""
    b = _bench_module()
    f = b.PROFILED["fma_share"]
    assert 0.0 < f < 1.0
    lvl = b.PROFILED["level"]
    assert b.mixed_ceiling(lvl, 20.0, 20.0, 39.1) == pytest.approx(min(20.0 / (1 - f), 20.0 / f, 39.1))
    # issue-bound when both pipes are fast
    assert b.mixed_ceiling(lvl, 1e6, 1e6, 39.1) == pytest.approx(39.1)
    # a pure ALU stream would be limited by the ALU rate alone
    assert b.mixed_ceiling(lvl, 20.0, 1e6, 1e6) == pytest.approx(20.0 / (1 - f))
    assert b.mixed_ceiling(lvl + 1, 20.0, 20.0, 39.1) is None


@pytest.mark.parametrize("flags,metric_tail,cfg_key", [
    (["--gap-open", "-2", "--gap-extend", "-1"], "affine-gap path", "path"),
    (["--matrix", "blosum62"], "substitution matrix (BLOSUM62 protein)", "matrix"),
])
def test_reference_line_other_paths(flags, metric_tail, cfg_key):
    """--impl reference times the oracle of the path the GPU arm runs for the
    same flags, under that arm's metric and config."""
    lines = run(["--impl", "reference", *flags, "--pairs", "100", "--steps", "1",
                 "--warmup", "0", "--cpu-seconds", "1"])
    assert len(lines) == 1
    j = lines[0]
    assert j["metric"].endswith(metric_tail) and j["value"] > 0
    assert cfg_key in j["config"] and "l2" in j["config"]
    assert j["cpu_baseline"]["value"] == j["value"]
