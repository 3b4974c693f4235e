"""bench.py --impl reference (the oracle timed on the host cores) keeps the
benchmark line's contract; it needs no GPU.  Other ranks of a multi-process
launch print nothing and exit 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                           "--n-mol", "2000"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "atom-steps/s"
    for k in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_nothing():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [x for x in r.stdout.splitlines() if x.startswith("{")]


def test_efficiency_against_eq21():
    sys.path.insert(0, ROOT)
    import bench

    fg = {"mean_list": 409.5, "mean_list_pruned": 304.3, "pair_ms_per_launch": 0.736, "ms_per_step": 1.05}
    e = bench.efficiency_eq21(fg, 0.162, 0.317, 85.8, 52.5)
    assert abs(e["n_star_walked"] - 52.5 / 304.3) < 1e-4 and abs(e["n_star_lists"] - 85.8 / 409.5) < 1e-4
    assert abs(e["eta_pair"] - 0.736 / 0.162) < 1e-3 and abs(e["eta_tot"] - 1.05 / 0.317) < 1e-3
    assert abs(e["chi_walked"] - e["eta_tot"] * e["n_star_walked"]) < 2e-3
    assert bench.efficiency_eq21({}, 0.1, 0.3, 1.0, 1.0) is None
