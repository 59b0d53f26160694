"""Host-side helpers of the benchmark (no GPU): the per-unit byte model of the roofline, the
kernel-launch count per traversal, the harmonic mean and the source check of recorded
DRAM traffic."""
import hashlib
import os

import pytest

import bench


def test_byte_models_follow_the_per_unit_figures():
    # bottom-up: N_core / 8 B bitmap (4 B per word), 16 B per unvisited vertex,
    # 4 B + 1 bit per entry examined, 8 B per vertex found
    lv = {"examined": 800, "discovered": 10}
    assert bench.bu_bytes(lv, n_core=1000, visited_before=200, nwords=32) == pytest.approx(
        4 * 32 + 16 * 800 + 4.125 * 800 + 8 * 10)
    # top-down: 16 B per frontier vertex, 8 B per frontier edge, 12 B per vertex found
    assert bench.td_bytes({"frontier": 3, "frontier_edges": 50, "discovered": 7}) == 16 * 3 + 8 * 50 + 12 * 7


def test_batch_byte_model_follows_the_per_unit_figures():
    work = {"pull_vertices": 10, "pull_entries": 100, "push_entries": 50, "discovered": 7}
    # one graph with 64 lanes, 1000 vertices, 400 core vertices (one lane word)
    assert bench.batch_bytes(work, [(64, 1000, 400)]) == pytest.approx(
        24 * 10 + 12 * 100 + 12 * 50 + 40 * 7 + 8 * 64 * 1000 + 384 * 400)
    # 65 lanes take two lane words
    assert bench.batch_bytes({k: 0 for k in work}, [(65, 10, 4)]) == pytest.approx(8 * 65 * 10 + 384 * 4 * 2)


def test_launch_count_per_traversal():
    # reset, start, anchors, output, fixup + per level one decide and the step kernels
    # (top-down 1, plus a queue rebuild after bottom-up; bottom-up gather + scan, or one
    # streaming kernel, plus a mark after top-down)
    trace = [{"direction": "td"}, {"direction": "bu"}, {"direction": "bu"}, {"direction": "td"}]
    assert bench.launches_of(trace) == 5 + 4 + 1 + 3 + 2 + 2
    trace = [{"direction": "td"}, {"direction": "bu", "stream": True}, {"direction": "bu", "stream": False}]
    assert bench.launches_of(trace) == 5 + 3 + 1 + 2 + 2


def test_harmonic_mean_ignores_non_positive():
    assert bench.hmean([2.0, 2.0]) == pytest.approx(2.0)
    assert bench.hmean([1.0, 3.0]) == pytest.approx(1.5)
    assert bench.hmean([0.0, -1.0]) == 0.0


def test_recorded_traffic_is_used_only_for_the_current_source():
    path = os.path.join(bench.ROOT, "profiles", "bfs_bu_traffic.txt")
    txt = open(path).read()
    src = open(os.path.join(bench.ROOT, "paper_2009_07463_gb300", "csrc", "bfs.cu"), "rb").read()
    current = hashlib.sha256(src).hexdigest()[:16] in txt
    got = bench.traffic_from_profiles("bfs_bu")
    assert (got is not None) == current
    if got is not None:
        assert got > 0


def test_reference_arm_prints_the_contract_line():
    # the reference arm times the CPU oracle; at a tiny scale it runs here without a GPU
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--scale", "10",
                        "--roots", "2", "--steps", "3", "--warmup", "3"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 3 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
