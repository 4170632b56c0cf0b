"""The benchmark's reference arm (the oracle, timed on the host cores) runs
without a GPU and prints the contract's JSON line; under torchrun only rank 0
prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--n", "300", "--density", "0.5", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    return [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_prints_one_line():
    lines = run({"RANK": "0"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["unit"] == "starts/s"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1)
    assert cb["value"] == d["value"]
    assert cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["n"] == 300


def test_reference_arm_other_ranks_print_nothing():
    assert run({"RANK": "1"}) == []


def test_all_cores_sample_does_the_single_thread_work():
    """The oracle sample spread over processes (evaluation and ascents in
    workers, screen and best-of over the whole batch) climbs exactly the starts
    the single-thread sample climbs, with the same flips."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    from paper_1706_00037_gb300 import synth
    a = argparse.Namespace(n=300, density=0.5, lam=0.5)
    op = bench.OraclePool(300, 0.5, 300)
    try:
        _, flips_all = bench.cpu_sample_all_cores(op, a, 200, 77)
    finally:
        op.close()
    _, flips_one = bench.cpu_sample(a, synth.make_instance(300, 0.5, 300), 200, 77)
    assert flips_all == flips_one > 0
