#!/usr/bin/env python
"""Benchmark: harmonic-mean GTEPS of edge-tree BFS over 64 roots on R-MAT scale 26.

One step = one single-root edge-tree BFS (gt_bfs) from each of the 64 seeded roots, each
timed on its own with CUDA events on the launching stream, inputs resident in HBM (the
graph is built once, untimed, as Graph500 excludes construction). GTEPS of a run = input
tuples with both ends reached / its time; value = harmonic mean over all timed runs
(times the number of replicas for N > 1: every GPU holds a full replica and takes its own
64 roots, so per-GPU work is fixed and scaling is weak).

Also measured, outside the timed region: the plain direction-optimizing BFS on the unsplit
graph (same roots), the end-to-end number through the C-ABI with host output buffers,
the roofline of the bottom-up kernel (durations from CUDA events around each launch in a
kernel-timing pass, algorithmic bytes from the per-level work counts), and the CPU oracle
on a bounded sample of the same workload.

--impl reference times the CPU oracle itself (serial BFS, the checker the tests use) on
the same workload, one root per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import re
import signal
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

E2E_CHUNK = 16  # roots per gt_bfs_roots call in the end-to-end pass
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e nominal bandwidth, reported beside the measured copy peak
METRIC = "harmonic-mean GTEPS over 64 roots at R-MAT scale 26; served queries/s and p99"
UNIT = "GTEPS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=26)
    ap.add_argument("--edgefactor", type=int, default=16)
    ap.add_argument("--roots", type=int, default=64)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--root-seed", type=int, default=2)
    ap.add_argument("--mh", type=int, default=0)
    ap.add_argument("--cpu-baseline", default="on", choices=["on", "off"])
    ap.add_argument("--cpu-roots", type=int, default=1)
    ap.add_argument("--no-extras", action="store_true", help="skip plain/e2e/roofline/batch/serve passes")
    ap.add_argument("--no-batch-serve", action="store_true", help="skip the short batch and serve passes")
    ap.add_argument("--trace-out", default="")
    ap.add_argument("--bu-hub-first", action="store_true",
                    help="degree-aware bottom-up (Alg. 3 probe order, min-id parents restored after the loop)")
    ap.add_argument("--alpha", type=int, default=0, help="top-down -> bottom-up switch constant (0: library default)")
    ap.add_argument("--no-plain", action="store_true",
                    help="build without the unsplit view (with --no-extras: less device memory, e.g. for profiling)")
    ap.add_argument("--root-list", default="", help="comma-separated roots instead of the seeded ones")
    ap.add_argument("--launch-mode", default="graph", choices=["graph", "host"],
                    help="host: one launch per kernel (lets ncu see every kernel; slower)")
    ap.add_argument("--workload", default="et", choices=["et", "batch", "serve", "study"],
                    help="et: single-root edge-tree BFS (the headline line); batch: 64-root lane words "
                         "on scale 24 plus a mixed 32-graph batch; serve: Poisson queries on 12 resident graphs; "
                         "study: scale / edge-factor / MH sweeps and the gain ablation, edge-tree vs plain")
    ap.add_argument("--batch-scale", type=int, default=24, help="batch workload: R-MAT scale of the 64-root part")
    ap.add_argument("--batch-parts", default="single,mixed", help="batch workload parts: single (one graph) and/or mixed")
    ap.add_argument("--no-batch-autotune", action="store_true", help="batch workload: keep default tuning")
    ap.add_argument("--study-scales", default="20,22,24,26,27")
    ap.add_argument("--study-efs", default="8,16,32")
    ap.add_argument("--study-mhs", default="0,1,2,-1")
    ap.add_argument("--study-roots", type=int, default=32)
    ap.add_argument("--serve-rates", default="4000,16000,48000")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-join-levels", type=int, default=-1,
                    help="level boundaries at which queries may join a running batched launch (-1: library default)")
    ap.add_argument("--serve-streams", type=int, default=4, help="server streams (flights at once)")
    ap.add_argument("--serve-policies", default="adaptive,batched,single",
                    help="server dispatch policies to run on each arrival schedule (the first is the headline)")
    return ap.parse_args()


def workload(a) -> dict:
    n = 1 << a.scale
    return {"workload": f"rmat_s{a.scale}_ef{a.edgefactor}_edge_tree_bfs", "scale": a.scale,
            "edgefactor": a.edgefactor, "n": n, "m": a.edgefactor * n, "roots": a.roots, "mh": a.mh,
            "initiator": [0.57, 0.19, 0.19, 0.05], "seed": a.seed, "root_seed": a.root_seed,
            "l2": "inputs larger than L2 (graph and core CSR are GBs; 129 MB L2)",
            "parallelism": "replicas"}


def hmean(x):
    x = [v for v in x if v > 0]
    return len(x) / sum(1.0 / v for v in x) if x else 0.0


# ---- CPU oracle leg (spawned process; never touches the GPU) -----------------------------

def oracle_job(scale, edgefactor, seed, root_seed, nroots, warm, q, go, save_dir=None):
    """Builds the oracle graph (untimed), then times serial oracle BFS from nroots roots.
    Waits for `go`, so its host memory traffic never overlaps the GPU's timed passes. With
    save_dir, the first root's levels and parents are saved there (level.npy, parent.npy)
    for an element-by-element comparison with the GPU's answer."""
    go.wait()
    try:
        import numpy as np

        import graphgen
        from oracle import OracleGraph, traversed_tuples
        n = 1 << scale
        t0 = time.time()
        e = graphgen.rmat_edges(scale, edgefactor, seed=seed)
        og = OracleGraph(e, n)
        setup = time.time() - t0
        roots = graphgen.pick_roots(root_seed, n, max(nroots, 1), og.degree())
        res = []
        for i in range(warm):
            og.bfs(int(roots[i % len(roots)]))
        for i, r in enumerate(roots[:nroots].tolist()):
            t = time.perf_counter()
            lv, pa = og.bfs(int(r))
            dt = time.perf_counter() - t
            res.append((int(r), dt, traversed_tuples(e, lv)))
            if i == 0 and save_dir:
                np.save(os.path.join(save_dir, "level.npy"), lv)
                np.save(os.path.join(save_dir, "parent.npy"), pa)
        q.put({"ok": True, "setup_s": setup, "runs": res})
    except Exception as ex:  # reported in the JSON line, never fatal
        q.put({"ok": False, "error": repr(ex)})


def start_oracle(a, nroots, warm, save_dir=None):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    go = ctx.Event()
    p = ctx.Process(target=oracle_job,
                    args=(a.scale, a.edgefactor, a.seed, a.root_seed, nroots, warm, q, go, save_dir), daemon=True)
    p.start()
    return p, q, go


def parity_obj(cfg_name, root, got_level, got_parent, save_dir) -> dict:
    """Element-by-element comparison of the GPU's answer for `root` with the oracle's."""
    import numpy as np
    try:
        wl = np.load(os.path.join(save_dir, "level.npy"))
        wp = np.load(os.path.join(save_dir, "parent.npy"))
    except Exception as ex:
        return {"config": cfg_name, "roots": 0, "equal": None, "error": repr(ex)}
    ml = int((wl != got_level).sum())
    mp_ = int((wp != got_parent).sum())
    return {"config": cfg_name, "roots": 1, "root": int(root), "vertices": int(wl.size), "equal": ml == 0 and mp_ == 0,
            "level_mismatches": ml, "parent_mismatches": mp_,
            "how": "levels and min-id parents of gt_bfs (device, edge-tree BFS) against the CPU oracle (serial BFS "
                   "on the unpeeled graph) from the same root, every vertex compared"}


def oracle_result(p, q, go, timeout):
    go.set()
    try:
        r = q.get(timeout=timeout)
    except Exception:
        r = {"ok": False, "error": "oracle leg timed out"}
    if p.is_alive():
        p.kill()
    return r


def cpu_baseline_obj(r, nroots):
    if not r.get("ok"):
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.get("error")}
    gteps = [m / dt / 1e9 for (_, dt, m) in r["runs"]]
    return {"value": hmean(gteps), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"serial oracle BFS (Alg. 1 top-down, min-id parents) from the first {nroots} of the "
                      f"same seeded roots on the same scale-26 graph; oracle graph built untimed "
                      f"({r['setup_s']:.0f} s with all host threads)",
            "seconds": [round(dt, 3) for (_, dt, _) in r["runs"]]}


# ---- clocks -------------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index: int):
        self.path = tempfile.mktemp(prefix="gt_clocks_", suffix=".csv")
        self.dev = dev_index
        self.p = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.send_signal(signal.SIGTERM)
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = []
        for ln in open(self.path):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = sorted(v for v in (num(r[1]) for r in rows) if v is not None)
        mx = max((v for v in (num(r[2]) for r in rows) if v is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ---- roofline helpers ---------------------------------------------------------------------

def bu_bytes(lv: dict, n_core: int, visited_before: int, nwords: int) -> float:
    """Algorithmic bytes of one bottom-up step, per-unit figures of the method: the visited
    bitmap once (N_core / 8 B), a 16 B row-offset pair per unvisited vertex, 4 B per
    adjacency entry examined plus its 1-bit frontier probe, 8 B (level, parent) per vertex
    found."""
    unvisited = n_core - visited_before
    return 4.0 * nwords + 16.0 * unvisited + 4.125 * lv["examined"] + 8.0 * lv["discovered"]


def td_bytes(lv: dict) -> float:
    """Top-down step: a 16 B row-offset pair per frontier vertex, 4 B per frontier edge read
    plus 4 B for the state check of the vertex it reaches, 12 B (level, parent, queue
    entry) per vertex found."""
    return 16.0 * lv["frontier"] + 8.0 * lv["frontier_edges"] + 12.0 * lv["discovered"]


def traffic_from_profiles(kernel: str) -> float | None:
    """ncu DRAM bytes per launch recorded under profiles/, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    src = open(os.path.join(ROOT, "paper_2009_07463_gb300", "csrc", "bfs.cu"), "rb").read()
    if not h or not b or h.group(1) != hashlib.sha256(src).hexdigest()[:16]:
        return None
    return float(b.group(1))


def launches_of(trace: list[dict]) -> int:
    """Kernels one gt_bfs launches: reset, start, per level the step kernels + decide, the
    anchor gather, output and the root-walk fix-up (resolve passes are absent at MH = 0 but
    for K2 tops). Step kernels: top-down 1, plus a queue rebuild after a bottom-up step;
    bottom-up over the gathered list 2 (gather, scan), streaming bottom-up 1, each plus a
    mark after a top-down step."""
    k = 5
    if not trace:
        return k + 2
    prev = None
    for t in trace:
        k += 1  # decide
        if t["direction"] == "td":
            k += 2 if prev == "bu" else 1
        else:
            k += (1 if t.get("stream") else 2) + (1 if prev == "td" else 0)
        prev = t["direction"]
    return k


# ---- replicas (N > 1): each rank holds a full graph and takes its own roots -------------

def rank_roots(all_roots, rank: int, per_rank: int) -> list[int]:
    """Rank r's share of the seeded roots: entries [r * per_rank, (r + 1) * per_rank)."""
    return [int(x) for x in all_roots[rank * per_rank:(rank + 1) * per_rank]]


def combine_ranks(ms_per_step: float, hm: float, dist, device):
    """Whole-job numbers: the slowest rank's time per step, and N x the harmonic mean of
    the ranks' GTEPS (N replicas run concurrently, each at its own rate). No data-path
    collective: this is the only exchange, after the timed region."""
    if dist is None:
        return ms_per_step, hm
    import torch
    world = dist.get_world_size()
    t = torch.tensor([ms_per_step, hm], dtype=torch.float64, device=device)
    gathered = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(gathered, t)
    return max(float(x[0]) for x in gathered), world * hmean([float(x[1]) for x in gathered])


# ---- main ---------------------------------------------------------------------------------

def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, world, rank)
    if a.workload == "batch":
        return run_batch_workload(a, rank, local)
    if a.workload == "serve":
        return run_serve_workload(a, rank, local)
    if a.workload == "study":
        return run_study_workload(a, rank, local)

    # the oracle leg is spawned before the first GPU call
    oracle = None
    oracle_dir = None
    if a.cpu_baseline == "on" and rank == 0 and world == 1:
        oracle_dir = tempfile.mkdtemp(prefix="gt_oracle_")
        oracle = start_oracle(a, a.cpu_roots, 0, oracle_dir)

    import numpy as np
    import torch

    import graphgen
    import paper_2009_07463_gb300 as gt

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n = 1 << a.scale
    m = a.edgefactor * n
    cfg = workload(a)

    # graph: device-resident tuples, built once (untimed)
    edges = torch.empty((m, 2), dtype=torch.int64, device=dev)
    graphgen.rmat_edges_device(edges.data_ptr(), a.scale, m, seed=a.seed, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.time()
    g = gt.gt_graph_build(edges, n, mh=a.mh, keep_plain=not (a.no_plain and a.no_extras), stream=stream)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    if a.launch_mode == "host":
        g.set_tuning(launch_mode=1)
    if a.alpha > 0:
        g.set_tuning(alpha=a.alpha)
    if a.bu_hub_first:
        g.set_tuning(bu_hub_first=1)
    st = g.stats()
    deg = g.degree()
    all_roots = graphgen.pick_roots(a.root_seed, n, a.roots * world, deg)
    roots = rank_roots(all_roots, rank, a.roots)
    if a.root_list:
        roots = [int(x) for x in a.root_list.split(",") if x]

    parent = torch.empty(n, dtype=torch.int32, device=dev)
    level = torch.empty(n, dtype=torch.int32, device=dev)

    # per-root TEPS numerator and level trace (untimed)
    tuples, traces = [], []
    for r in roots:
        g.bfs(r, parent, level, stream=stream)
        traces.append(g.trace())
        tuples.append(gt.gt_count_traversed(edges, level, stream=stream))

    def one_step(fn, record):
        evs = []
        for r in roots:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(r, parent, level, stream=stream)
            e1.record(stream)
            evs.append((e0, e1))
        if record is not None:
            record.append(evs)

    for _ in range(a.warmup):
        one_step(g.bfs, None)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    tstart = torch.cuda.Event(enable_timing=True)
    tend = torch.cuda.Event(enable_timing=True)
    rec = []
    tstart.record(stream)
    for _ in range(a.steps):
        one_step(g.bfs, rec)
    tend.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = tstart.elapsed_time(tend)
    run_ms = [[e0.elapsed_time(e1) for (e0, e1) in step] for step in rec]
    gteps = [tuples[i] / (ms * 1e-3) / 1e9 for step in run_ms for i, ms in enumerate(step)]
    hm = hmean(gteps)
    am = sum(gteps) / len(gteps)
    ms_per_step = total_ms / a.steps
    ms_per_step, value = combine_ranks(ms_per_step, hm, dist, dev)
    launches_per_step = sum(launches_of(tr) for tr in traces)

    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": cfg,
           "gpu_launches": launches_per_step * a.steps, "clocks": clk,
           "gteps_arith_mean": round(am, 3),
           "graph": {"nnz": st["nnz"], "n_core": st["n_core"], "nnz_core": st["nnz_core"],
                     "classes_CI_CE_TI_TL_VZ": st["n_class"], "build_s": round(build_s, 2),
                     "device_gb": round(st["device_bytes"] / 1e9, 2)}}

    if not a.no_extras:
        # (a) plain direction-optimizing BFS on the unsplit graph, same roots, same timing
        for _ in range(1):
            one_step(g.bfs_plain, None)
        prec = []
        one_step(g.bfs_plain, prec)
        torch.cuda.synchronize()
        pg = [tuples[i] / (e0.elapsed_time(e1) * 1e-3) / 1e9 for i, (e0, e1) in enumerate(prec[0])]
        out["plain_do_bfs"] = {"value": round(hmean(pg), 3), "unit": UNIT,
                               "et_over_plain": round(hm / hmean(pg), 3) if hmean(pg) else None}

        # end to end through the C-ABI: host (pinned) output buffers, copies inside the timing.
        # gt_bfs_roots takes E2E_CHUNK roots per call, each with its own host buffers, and
        # overlaps the copy of one result with the traversal of the next
        hb = [(torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory())
              for _ in range(E2E_CHUNK)]
        g.bfs_roots(roots[:E2E_CHUNK], [b[0] for b in hb], [b[1] for b in hb], stream=stream)  # first use: staging
        e_time, e_tup = 0.0, 0.0
        for c0 in range(0, len(roots), E2E_CHUNK):
            chunk = roots[c0:c0 + E2E_CHUNK]
            t = time.perf_counter()
            g.bfs_roots(chunk, [b[0] for b in hb[:len(chunk)]], [b[1] for b in hb[:len(chunk)]], stream=stream)
            e_time += time.perf_counter() - t  # returns once every result is in host memory
            e_tup += sum(tuples[c0:c0 + len(chunk)])
        hp, hl = hb[0]
        g.bfs(roots[0], hp, hl, stream=stream)
        eg = []
        for i, r in enumerate(roots):
            t = time.perf_counter()
            g.bfs(r, hp, hl, stream=stream)  # returns once the results are in host memory
            eg.append(tuples[i] / (time.perf_counter() - t) / 1e9)
        # the host link itself: copy-engine device -> host rate into one pinned pair
        db = torch.empty(2 * n, dtype=torch.int32, device=dev)
        hb2 = torch.empty(2 * n, dtype=torch.int32).pin_memory()
        hb2.copy_(db, non_blocking=True)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        for _ in range(3):
            hb2.copy_(db, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        link_gbs = 3 * 8 * n / (c0.elapsed_time(c1) * 1e-3) / 1e9
        del db, hb2
        out["e2e"] = {"value": round(e_tup / e_time / 1e9, 3), "unit": UNIT, "h2d_bytes_per_step": 8 * len(roots),
                      "d2h_bytes_per_step": 8 * n * len(roots),
                      "how": f"gt_bfs_roots, {E2E_CHUNK} roots per call into pinned host parent/level buffers (one "
                             "pair per root); host clock around each call, which returns once every result is in "
                             "host memory; traversed tuples / summed call time",
                      "single_call": {"value": round(hmean(eg), 3),
                                      "how": "gt_bfs per root into one pinned pair (returns after its copy); "
                                             "harmonic mean"},
                      "link_d2h_gbs_copy_engine": round(link_gbs, 1),
                      "link_bound_gteps": round(sum(tuples) / len(tuples) / (8 * n / (link_gbs * 1e9)) / 1e9, 1)}

        # roofline of the bottom-up kernel: work counts, then CUDA-event durations per launch
        g.set_tuning(count_work=1, launch_mode=1)
        counted = []
        for r in roots:
            g.bfs(r, parent, level, stream=stream)
            counted.append(g.trace())
        g.set_tuning(count_work=0, launch_mode=1, time_kernels=1)
        timed = []
        for r in roots:
            g.bfs(r, parent, level, stream=stream)
            timed.append(g.trace())
        g.set_tuning(count_work=0, launch_mode=1 if a.launch_mode == "host" else 0, time_kernels=1)
        phases = []
        for r in roots:
            g.bfs(r, parent, level, stream=stream)
            phases.append(g.timing())
        g.set_tuning(time_kernels=0)
        out["phases_ms_mean"] = {k: round(sum(p[k] for p in phases) / len(phases), 4) for k in phases[0]}
        nc = st["n_core"]
        nwords = -(-max(nc, 1) // 32)
        nwords = -(-nwords // 128) * 128
        bu_b = bu_t = td_b = td_t = 0.0
        bu_n = td_n = 0
        for cw, tm in zip(counted, timed):
            visited = 1
            for lc, lt in zip(cw, tm):
                if lc["direction"] == "bu":
                    bu_b += bu_bytes(lc, nc, visited, nwords)
                    bu_t += lt["step_ms"]
                    bu_n += 1
                else:
                    td_b += td_bytes(lc)
                    td_t += lt["step_ms"]
                    td_n += 1
                visited += lc["discovered"]
        import json as _j
        peaks = _j.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        peak = peaks.get("hbm_gbs", 6800.0)
        peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
        bu_gbs = bu_b / (bu_t * 1e-3) / 1e9 if bu_t > 0 else 0.0
        td_gbs = td_b / (td_t * 1e-3) / 1e9 if td_t > 0 else 0.0
        trf = traffic_from_profiles("bfs_bu")
        out["roofline"] = {"bound": "hbm", "kernel": "bottom-up step (bfs_mark, bfs_bu_stream; bfs_bu_gather + bfs_bu_scan)",
                           "achieved": round(bu_gbs, 1), "peak": peak,
                           "peak_source": peak_src, "unit": "GB/s", "frac": round(bu_gbs / peak, 4),
                           "peak_nominal": HBM_NOMINAL_GBS, "frac_nominal": round(bu_gbs / HBM_NOMINAL_GBS, 4),
                           "traffic": trf, "launches": bu_n,
                           "dram_achieved": round(trf / (bu_t / max(bu_n, 1) * 1e-3) / 1e9, 1) if trf and bu_t > 0 else None,
                           "dram_frac": round(trf / (bu_t / max(bu_n, 1) * 1e-3) / 1e9 / peak, 4) if trf and bu_t > 0 else None,
                           "bytes_per_launch": round(bu_b / max(bu_n, 1)),
                           "ms_per_launch": round(bu_t / max(bu_n, 1), 4),
                           "share_of_step_time": round(bu_t / (bu_t + td_t), 3) if bu_t + td_t > 0 else None,
                           "td": {"achieved": round(td_gbs, 1), "frac": round(td_gbs / peak, 4), "launches": td_n,
                                  "ms_per_launch": round(td_t / max(td_n, 1), 4)},
                           "how": "achieved = algorithmic bytes from per-level work counts / kernel duration from "
                                  "CUDA events around each launch (host-driven kernel-timing pass, same roots); "
                                  "dram_achieved = ncu DRAM bytes per bottom-up step (profiles/bfs_bu_traffic.txt, "
                                  "same kernel source) / the same duration"}
        if a.trace_out:
            json.dump({"roots": roots, "counted": counted, "timed": timed, "tuples": tuples,
                       "run_ms": run_ms, "phases": phases}, open(a.trace_out, "w"))

        # the other half of the metric: batched and served queries/s (short passes)
        if not a.no_batch_serve and rank == 0:
            out["batch"] = batch_summary(batch_measure(a, gt, graphgen, torch, dev, ["single", "mixed"], True))
            out["serve"] = serve_summary(a, serve_measure(gt, graphgen, torch, dev, [1000.0, 4000.0, 16000.0], 1.5,
                                                          ["adaptive"], -1, a.serve_streams))
            torch.cuda.empty_cache()

    if oracle is not None:
        # every GPU pass is done: the CPU leg starts now (its graph build takes all host
        # threads, which would disturb the host side of the passes above)
        out["cpu_baseline"] = cpu_baseline_obj(oracle_result(*oracle, timeout=1800), a.cpu_roots)
        if out["cpu_baseline"]["value"]:
            out["cpu_baseline"]["cores"] = 1
            # the same root through gt_bfs, compared with the oracle's answer element by element
            g.bfs(roots[0], parent, level, stream=stream)
            torch.cuda.synchronize()
            out["parity"] = parity_obj(cfg["workload"], roots[0], level.cpu().numpy(), parent.cpu().numpy(), oracle_dir)
        for f in ("level.npy", "parent.npy"):
            try:
                os.unlink(os.path.join(oracle_dir, f))
            except OSError:
                pass
        try:
            os.rmdir(oracle_dir)
        except OSError:
            pass
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_reference(a, world, rank):
    """The CPU oracle timed as the reference arm, one seeded root per step on the same graph
    (built untimed). The W + K roots run concurrently on the host cores, one serial oracle
    BFS per thread (the C oracle releases the GIL), so the whole run takes about two root
    times instead of W + K; each step's GTEPS comes from its own root's time."""
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor

    import graphgen
    from oracle import OracleGraph, traversed_tuples
    n = 1 << a.scale
    t0 = time.time()
    e = graphgen.rmat_edges(a.scale, a.edgefactor, seed=a.seed)
    og = OracleGraph(e, n)
    setup = time.time() - t0
    roots = graphgen.pick_roots(a.root_seed, n, a.roots, og.degree()).tolist()
    cores = max(1, min(len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1),
                       a.warmup + a.steps))

    def one(i):
        r = roots[i % len(roots)]
        t = time.perf_counter()
        lv, _ = og.bfs(r)
        dt = time.perf_counter() - t
        return i, dt, traversed_tuples(e, lv) if i >= a.warmup else 0

    tt = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        done = list(ex.map(one, range(a.warmup + a.steps)))
    wall = time.perf_counter() - tt
    runs = [m / dt / 1e9 for (i, dt, m) in done if i >= a.warmup]
    secs = [dt for (i, dt, m) in done if i >= a.warmup]
    v = hmean(runs)
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(1e3 * sum(secs) / len(secs), 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
           "data": "synthetic", "config": workload(a),
           "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"one seeded root per step on the same scale-{a.scale} graph (warm-up and "
                                      f"timed roots together, {cores} at a time, one serial oracle BFS per host "
                                      f"thread; each step timed on its own thread); oracle graph built untimed "
                                      f"in {setup:.0f} s",
                            "wall_s": round(wall, 1),
                            "aggregate_gteps": round(sum(m for (i, _, m) in done if i >= a.warmup) / 1e9 / wall, 4)},
           "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---- batched and served workloads -------------------------------------------------------

def _make_graph(gt, graphgen, torch, kind, a_, seed, dev):
    """R-MAT (kind 'rmat', a_ = scale, edge factor 16) or uniform (a_ = (n, avg degree))."""
    if kind == "rmat":
        n, m = 1 << a_, 16 << a_
        e = torch.empty((m, 2), dtype=torch.int64, device=dev)
        graphgen.rmat_edges_device(e.data_ptr(), a_, m, seed=seed)
    else:
        n, d = a_
        m = n * d // 2
        e = torch.empty((m, 2), dtype=torch.int64, device=dev)
        graphgen.uniform_edges_device(e.data_ptr(), n, m, seed=seed)
    torch.cuda.synchronize()
    g = gt.gt_graph_build(e, n)
    return g, e


def batch_measure(a, gt, graphgen, torch, dev, parts, autotune) -> dict:
    """Batched launches against the same roots one at a time (gt_bfs): R-MAT scale
    a.batch_scale with 64 roots in one lane word ("single"), and 32 mixed graphs (R-MAT
    scales 14-22, uniform graphs of average degree 16) with 64 roots each ("mixed")."""
    res = {}

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def measure(specs, label):
        graphs, roots, tuples = [], [], []
        for i, (kind, arg) in enumerate(specs):
            g, e = _make_graph(gt, graphgen, torch, kind, arg, 100 + i, dev)
            if autotune:
                g.autotune(nsample=4, seed=7)
            r = graphgen.pick_roots(3 + i, g.n, 64, g.degree()).tolist()
            lv = torch.empty(g.n, dtype=torch.int32, device=dev)
            pa = torch.empty(g.n, dtype=torch.int32, device=dev)
            tt = []
            for x in r:
                g.bfs(x, pa, lv)
                tt.append(gt.gt_count_traversed(e, lv))
            del e
            graphs.append(g)
            roots.append(r)
            tuples.append(tt)
        outs_p = [torch.empty((64, g.n), dtype=torch.int32, device=dev) for g in graphs]
        outs_l = [torch.empty((64, g.n), dtype=torch.int32, device=dev) for g in graphs]
        ms_batch = timed(lambda: gt.gt_bfs_batch(graphs, roots, outs_p, outs_l), 3)
        work = gt.gt_bfs_batch_work(graphs[0])
        bb = batch_bytes(work, [(len(r), g.n, g.stats()["n_core"]) for g, r in zip(graphs, roots)])
        lv = torch.empty(max(g.n for g in graphs), dtype=torch.int32, device=dev)
        pa = torch.empty_like(lv)

        def seq():
            for g, r in zip(graphs, roots):
                for x in r:
                    g.bfs(x, pa[:g.n], lv[:g.n])
        ms_seq = timed(seq, 1)
        nq = sum(len(r) for r in roots)
        te = sum(sum(t) for t in tuples)
        res[label] = {"queries": nq, "batch_ms": round(ms_batch, 3), "sequential_ms": round(ms_seq, 3),
                      "batch_qps": round(nq / ms_batch * 1e3, 1), "sequential_qps": round(nq / ms_seq * 1e3, 1),
                      "batch_gteps_equiv": round(te / ms_batch / 1e6, 1),
                      "sequential_gteps_equiv": round(te / ms_seq / 1e6, 1),
                      "speedup": round(ms_seq / ms_batch, 2),
                      "roofline": {"bound": "hbm", "kernel": "batched launch (batch_run + output passes)",
                                   "achieved": round(bb / (ms_batch * 1e-3) / 1e9, 1), "peak": hbm_peak()[0],
                                   "unit": "GB/s", "frac": round(bb / (ms_batch * 1e-3) / 1e9 / hbm_peak()[0], 4),
                                   "bytes_per_launch": round(bb), "work": work}}
        del outs_p, outs_l
        for g in graphs:
            g.free()
        torch.cuda.empty_cache()

    if "single" in parts:
        measure([("rmat", a.batch_scale)], f"rmat_s{a.batch_scale}_64_roots")
    if "mixed" in parts:
        mixed = [("rmat", 14 + (i % 9)) for i in range(24)] + [("uniform", (1 << (15 + (i % 6)), 16)) for i in range(8)]
        measure(mixed, "mixed_32_graphs_64_roots_each")
    return res


def batch_bytes(work: dict, graphs: list) -> float:
    """Algorithmic bytes of one batched launch, per-unit figures of the lane-word method:
    pull: 24 B per core vertex scanned (row-offset pair, visit word) + 12 B per adjacency
    entry read (entry, frontier word of the neighbour); push: 12 B per entry read (entry,
    visit word of the target); commit: 40 B per vertex discovered in a lane word (next
    frontier word, visit word read and written, row-offset pair); output: 8 B per lane and
    vertex written (level, parent) + 384 B per core vertex and lane word read (the staged
    rows, 64 x (4 B parent + 2 B level)). graphs: (lanes, n, n_core) per graph."""
    b = 24.0 * work["pull_vertices"] + 12.0 * work["pull_entries"] + 12.0 * work["push_entries"]
    b += 40.0 * work["discovered"]
    for lanes, n, nc in graphs:
        b += 8.0 * lanes * n + 384.0 * nc * ((lanes + 63) // 64)
    return b


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)).get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def batch_summary(res: dict) -> dict:
    return {"unit": "queries/s", "autotuned": True,
            "parts": {k: {x: v[x] for x in ("queries", "batch_qps", "sequential_qps", "batch_ms", "sequential_ms",
                                            "speedup", "roofline")} for k, v in res.items()},
            "how": "gt_bfs_batch (64-root lane words, one persistent launch, captured CUDA graph, autotuned) "
                   "against the same roots one gt_bfs call at a time; CUDA events, mean of 3 launches"}


def run_batch_workload(a, rank, local):
    """Batch workload: 64 roots in one lane word on R-MAT scale 24 (--batch-scale), and a mixed batch of 32 graphs
    (R-MAT scales 14-22, uniform graphs of average degree 16), 64 roots each, every batch in
    one persistent launch with autotuned parameters; against the same roots run one at a
    time with gt_bfs. Queries/s and GTEPS-equivalent (traversed tuples / time)."""
    import torch

    import graphgen
    import paper_2009_07463_gb300 as gt
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    parts = [x for x in a.batch_parts.split(",") if x]
    res = batch_measure(a, gt, graphgen, torch, dev, parts, not a.no_batch_autotune)
    head = res.get("mixed_32_graphs_64_roots_each") or next(iter(res.values()))
    out = {"metric": "batched BFS queries/s (64-root lane words, one persistent launch)",
           "value": head["batch_qps"], "unit": "queries/s", "n_gpus": 1,
           "higher_is_better": True, "dtype": "int32", "data": "synthetic",
           "config": {"workload": f"batch: rmat s{a.batch_scale} x 64 roots; 32 mixed graphs (rmat s14-22, uniform "
                                  "deg 16) x 64 roots", "parts": parts, "autotuned": not a.no_batch_autotune,
                      "cuda_graph": "each batched launch is one captured graph, replayed"}, "results": res}
    print(json.dumps(out), flush=True)


def _serve_once(gt, graphs, bufs, RING, nq, gaps, gsel, roots, policy, join_levels=-1, streams=2):
    """One arrival schedule through a server with the given dispatch policy."""
    import threading
    srv = gt.Server(hbm_budget_bytes=48 << 30, streams=streams, max_batch_roots=128, window_us=100, policy=policy,
                    join_levels=None if join_levels < 0 else join_levels)
    gids = [srv.add_graph(g) for g in graphs]
    slot_busy = [[None] * RING for _ in graphs]
    ring_pos = [0] * len(graphs)
    lat = [0.0] * nq
    t_arr = [0.0] * nq
    tickets = [None] * nq
    done_ev = threading.Event()

    def collector():
        for j in range(nq):
            while tickets[j] is None:
                time.sleep(0.00005)
            srv.poll(tickets[j], 60000)
            lat[j] = time.perf_counter() - t_arr[j]
        done_ev.set()
    col = threading.Thread(target=collector)
    col.start()
    t0 = time.perf_counter()
    t_next = t0
    for j in range(nq):
        t_next += gaps[j]
        while time.perf_counter() < t_next:
            pass
        gi = int(gsel[j])
        k = ring_pos[gi]
        ring_pos[gi] = (k + 1) % RING
        prev = slot_busy[gi][k]
        if prev is not None:
            while lat[prev] == 0.0:  # ring buffer still owned by an earlier query
                time.sleep(0.00002)
        slot_busy[gi][k] = j
        t_arr[j] = t_next
        p, l = bufs[gi][k]
        tickets[j] = srv.submit(gids[gi], roots[j], p, l)
    done_ev.wait()
    st = srv.stats()  # latency stamped by the completion callback: submit -> results ready
    srv.destroy()
    col.join()
    return {"qps": round(st["qps"], 1), "p50_us": round(st["p50_us"], 1), "p99_us": round(st["p99_us"], 1),
            "batched_launches": st["batches"], "joined": st["joined"], "early": st["early"]}


def serve_measure(gt, graphgen, torch, dev, rates, seconds, policies, join_levels, streams) -> list:
    """12 resident graphs (R-MAT scales 18-25 at edge factor 16; uniform graphs of 2^20
    vertices and average degree 8-32), a 48 GiB HBM budget, Poisson arrivals of single-root
    queries at each rate (roots uniform over vertices of degree >= 1 of a uniformly chosen
    graph), served under each dispatch policy and run by one worker with sequential gt_bfs
    calls on the same schedule."""
    import numpy as np
    specs = [("rmat", s) for s in range(18, 26)] + [("uniform", (1 << 20, d)) for d in (8, 16, 24, 32)]
    graphs, cand = [], []
    for i, (kind, arg) in enumerate(specs):
        g, e = _make_graph(gt, graphgen, torch, kind, arg, 200 + i, dev)
        del e
        graphs.append(g)
        cand.append(np.flatnonzero(g.degree() > 0))
    torch.cuda.empty_cache()
    RING = 64
    bufs = [[(torch.empty(g.n, dtype=torch.int32, device=dev), torch.empty(g.n, dtype=torch.int32, device=dev))
             for _ in range(RING)] for g in graphs]
    rng = np.random.default_rng(11)
    results = []
    for rate in rates:
        nq = int(rate * seconds)
        gaps = rng.exponential(1.0 / rate, size=nq)
        gsel = rng.integers(0, len(graphs), size=nq)
        roots = [int(cand[gi][rng.integers(0, cand[gi].size)]) for gi in gsel]
        served = {}
        for pol in policies:
            served[pol] = _serve_once(gt, graphs, bufs, RING, nq, gaps, gsel, roots,
                                      {"adaptive": gt.GT_SERVE_ADAPTIVE, "batched": gt.GT_SERVE_BATCHED,
                                       "single": gt.GT_SERVE_SINGLE}[pol], join_levels, streams)
        # sequential single-root calls on the same schedule (one worker, FIFO)
        lat2 = []
        stream = torch.cuda.current_stream()
        t0 = time.perf_counter()
        t_arr2 = t0
        for j in range(nq):
            t_arr2 += gaps[j]
            now = time.perf_counter()
            if now < t_arr2:
                while time.perf_counter() < t_arr2:
                    pass
            gi = int(gsel[j])
            p, l = bufs[gi][j % RING]
            graphs[gi].bfs(roots[j], p, l, stream=stream)
            stream.synchronize()
            lat2.append(time.perf_counter() - t_arr2)
        t_end2 = t_arr2 + lat2[-1]
        lat2s = sorted(lat2)
        seq = {"qps": round(nq / (t_end2 - t0), 1), "p50_us": round(1e6 * lat2s[nq // 2], 1),
               "p99_us": round(1e6 * lat2s[min(nq - 1, int(0.99 * nq))], 1)}
        results.append({"rate_qps": rate, "queries": nq, "served": served, "sequential": seq})
    del bufs
    for g in graphs:
        g.free()
    torch.cuda.empty_cache()
    return results


def serve_summary(a, results) -> dict:
    pol = next(iter(results[0]["served"]))
    return {"unit": "queries/s", "policy": pol, "streams": a.serve_streams, "hbm_budget_gib": 48,
            "graphs": "12 resident: rmat s18-25 ef16, uniform 2^20 deg 8/16/24/32",
            "rates": [{"offered_qps": r["rate_qps"], "queries": r["queries"], "served_qps": r["served"][pol]["qps"],
                       "p50_us": r["served"][pol]["p50_us"], "p99_us": r["served"][pol]["p99_us"],
                       "sequential": r["sequential"]} for r in results],
            "how": "Poisson arrivals of single-root queries; latency = arrival -> results in the caller's device "
                   "buffers; sequential = one worker calling gt_bfs per query on the same schedule"}


def run_serve_workload(a, rank, local):
    """Serving workload (see serve_measure) at each --serve-rates rate under each
    --serve-policies policy, against sequential gt_bfs calls on the same schedule."""
    import torch

    import graphgen
    import paper_2009_07463_gb300 as gt
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rates = [float(x) for x in a.serve_rates.split(",") if x]
    policies = [x for x in a.serve_policies.split(",") if x]
    results = serve_measure(gt, graphgen, torch, dev, rates, a.serve_seconds, policies, a.serve_join_levels,
                            a.serve_streams)
    head = policies[0]
    best = max(results, key=lambda r: r["served"][head]["qps"])
    out = {"metric": "served BFS queries/s and p99 latency (continuous batching)", "value": best["served"][head]["qps"],
           "unit": "queries/s", "p99_us": best["served"][head]["p99_us"], "policy": head, "n_gpus": 1, "higher_is_better": True,
           "dtype": "int32", "data": "synthetic",
           "config": {"workload": "serve: 12 resident graphs (rmat s18-25 ef16, uniform 2^20 deg 8/16/24/32), "
                                  "Poisson arrivals", "hbm_budget_gib": 48, "streams": a.serve_streams, "max_batch_roots": 128,
                      "window_us": 100, "seconds_per_rate": a.serve_seconds},
           "rates": results}
    print(json.dumps(out), flush=True)


def run_study_workload(a, rank, local):
    """Sweeps and ablation around the headline (edge-tree vs plain direction-optimizing BFS,
    harmonic-mean GTEPS over the first --study-roots seeded roots, each root timed alone with
    CUDA events after one warm-up pass):
      scales   R-MAT scales --study-scales at edge factor 16, MH = 0;
      efs      edge factors --study-efs at --scale;
      mhs      maximum tree heights --study-mhs at --scale, edge factor 16 (class counts,
               tree height, build time beside the GTEPS);
      ablation at --scale: plain BFS; plain BFS after dropping zero-degree vertices (ids
               relabelled in order); the core BFS alone (root mapping + level loop, no
               edge-tree resolution or output pass: timing only); full edge-tree BFS."""
    import numpy as np
    import torch

    import graphgen
    import paper_2009_07463_gb300 as gt
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    nroots = a.study_roots

    def make(scale, ef, mh):
        n, m = 1 << scale, ef << scale
        e = torch.empty((m, 2), dtype=torch.int64, device=dev)
        graphgen.rmat_edges_device(e.data_ptr(), scale, m, seed=a.seed, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.time()
        g = gt.gt_graph_build(e, n, mh=mh, stream=stream)
        torch.cuda.synchronize()
        return g, e, n, time.time() - t0

    def timed(fn, roots, tuples, n):
        p = torch.empty(n, dtype=torch.int32, device=dev)
        l = torch.empty(n, dtype=torch.int32, device=dev)
        for r in roots:  # warm-up
            fn(r, p, l, stream=stream)
        evs = []
        for r in roots:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(r, p, l, stream=stream)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = [x.elapsed_time(y) for x, y in evs]
        return round(hmean([t / (x * 1e-3) / 1e9 for t, x in zip(tuples, ms)]), 2)

    def et_vs_plain(scale, ef, mh):
        g, e, n, build_s = make(scale, ef, mh)
        roots = graphgen.pick_roots(a.root_seed, n, nroots, g.degree()).tolist()
        lvl = torch.empty(n, dtype=torch.int32, device=dev)
        par = torch.empty(n, dtype=torch.int32, device=dev)
        tuples = []
        for r in roots:
            g.bfs(r, par, lvl, stream=stream)
            tuples.append(gt.gt_count_traversed(e, lvl, stream=stream))
        st = g.stats()
        out = {"scale": scale, "edgefactor": ef, "mh": mh, "et_gteps": timed(g.bfs, roots, tuples, n),
               "plain_gteps": timed(g.bfs_plain, roots, tuples, n), "core_fraction": round(st["n_core"] / n, 4),
               "classes_CI_CE_TI_TL_VZ": st["n_class"], "tree_height": st["height"], "build_s": round(build_s, 3)}
        out["et_over_plain"] = round(out["et_gteps"] / out["plain_gteps"], 3) if out["plain_gteps"] else None
        return g, e, n, roots, tuples, out

    res = {"scales": [], "efs": [], "mhs": []}
    for sc in [int(x) for x in a.study_scales.split(",") if x]:
        g, e, *_, out = et_vs_plain(sc, 16, 0)
        res["scales"].append(out)
        print(json.dumps({"study": "scale", **out}), flush=True)
        del g, e
        torch.cuda.empty_cache()
    for ef in [int(x) for x in a.study_efs.split(",") if x]:
        g, e, *_, out = et_vs_plain(a.scale, ef, 0)
        res["efs"].append(out)
        print(json.dumps({"study": "edgefactor", **out}), flush=True)
        del g, e
        torch.cuda.empty_cache()
    for mh in [int(x) for x in a.study_mhs.split(",") if x]:
        g, e, *_, out = et_vs_plain(a.scale, 16, mh)
        res["mhs"].append(out)
        print(json.dumps({"study": "mh", **out}), flush=True)
        del g, e
        torch.cuda.empty_cache()
    # ablation (Fig. 5): plain -> plain without zero-degree vertices -> core BFS alone -> full
    g, e, n, roots, tuples, full = et_vs_plain(a.scale, 16, 0)
    keep = torch.from_numpy(g.degree() > 0).to(dev)
    newid = torch.cumsum(keep.to(torch.int64), 0) - 1
    n2 = int(keep.sum().item())
    e2 = newid[e]
    g2 = gt.gt_graph_build(e2, n2, stream=stream)
    del e2
    torch.cuda.empty_cache()
    roots2 = newid[torch.tensor(roots, device=dev)].tolist()
    rmzero = timed(g2.bfs_plain, roots2, tuples, n2)
    g2.free()
    g.set_tuning(time_kernels=1)
    p = torch.empty(n, dtype=torch.int32, device=dev)
    lv = torch.empty(n, dtype=torch.int32, device=dev)
    core_ms = []
    for r in roots:
        g.bfs(r, p, lv, stream=stream)
    for r in roots:
        g.bfs(r, p, lv, stream=stream)
        t = g.timing()
        core_ms.append(t["start_ms"] + t["loop_ms"])
    g.set_tuning(time_kernels=0)
    core_only = round(hmean([t / (x * 1e-3) / 1e9 for t, x in zip(tuples, core_ms)]), 2)
    abl = {"scale": a.scale, "plain_gteps": full["plain_gteps"], "plain_without_zero_degree_gteps": rmzero,
           "core_bfs_only_gteps": core_only, "edge_tree_bfs_gteps": full["et_gteps"],
           "note": "core BFS alone = root mapping + level loop without resolution or output (timing only)"}
    res["ablation"] = abl
    print(json.dumps({"study": "ablation", **abl}), flush=True)
    out = {"metric": "edge-tree vs plain BFS, harmonic-mean GTEPS (sweeps and ablation)", "value": full["et_gteps"],
           "unit": "GTEPS", "n_gpus": 1, "higher_is_better": True, "dtype": "int32", "data": "synthetic",
           "config": {"workload": "study: R-MAT scale / edge factor / MH sweeps and the gain ablation",
                      "roots": nroots, "scale": a.scale}, "study": res}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
