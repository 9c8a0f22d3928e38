"""bench.py's contract pieces that need no GPU: the reference arm (the
oracle on host cores) prints one JSON line with the contract's keys, ranks
other than 0 print nothing, and the gradient kernel's committed ncu figures
belong to the kernel's current sources (the benchmark only quotes them
then)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "1", "--crop", "12"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["metric"] == bench.METRIC and d["unit"] == "vertices/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "vertices/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "1", "--crop", "12"],
             {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_gradient_profile_figures_match_the_kernel_sources():
    """The figures line of the gradient kernel's ncu summary names the hash
    of the sources it was taken on; a change to those sources needs a new
    capture (until then the benchmark reports no traffic and no issue fill)."""
    fig = bench.profile_figures()
    assert fig is not None, "the gradient kernel's summary has no figures for these sources"
    assert fig["warp_inst_per_vertex"] > 0 and fig["dram_bytes_per_vertex"] > 0
    r = _run(["--source-hash"])
    assert r.returncode == 0
    assert r.stdout.strip() == bench.kernel_source_hash()
