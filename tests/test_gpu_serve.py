"""Serving with continuous batching through the C-ABI: queries arriving from several
threads at random times over several resident graphs; every result must equal the
single-root answer (alone) bit for bit, and the server's host-side failure paths answer
with status codes (no GPU fault is ever provoked)."""
import random
import threading
import time

import numpy as np
import pytest

import graphgen
import paper_2009_07463_gb300 as gt
from oracle import OracleGraph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def graphs():
    out = []
    for i, (kind, a) in enumerate([("rmat", 12), ("rmat", 14), ("uniform", 30000), ("rmat", 10)]):
        if kind == "rmat":
            n = 1 << a
            e = graphgen.rmat_edges(a, 16, seed=70 + i)
        else:
            n = a
            e = graphgen.uniform_edges(n, n * 8, seed=70 + i)
        g = gt.gt_graph_build(e, n, mh=[0, 1, 0, -1][i])
        out.append((g, OracleGraph(e, n)))
    return out


@pytest.mark.parametrize("policy", [gt.GT_SERVE_ADAPTIVE, gt.GT_SERVE_BATCHED, gt.GT_SERVE_SINGLE])
def test_results_same_alone_and_in_the_mix(torch, graphs, policy):
    srv = gt.Server(streams=2, max_batch_roots=128, window_us=300, policy=policy)
    gids = [srv.add_graph(g) for g, _ in graphs]
    rng = random.Random(5)
    jobs = []
    for k in range(240):
        gi = rng.randrange(len(graphs))
        g, og = graphs[gi]
        deg = og.degree()
        root = rng.randrange(g.n)
        jobs.append((gi, root))
    bufs = [(torch.full((graphs[gi][0].n,), -7, dtype=torch.int32, device="cuda"),
             torch.full((graphs[gi][0].n,), -7, dtype=torch.int32, device="cuda")) for gi, _ in jobs]
    torch.cuda.synchronize()
    tickets = [None] * len(jobs)

    def producer(idx):
        for j in idx:
            gi, root = jobs[j]
            tickets[j] = srv.submit(gids[gi], root, bufs[j][0], bufs[j][1])
            time.sleep(rng.random() * 0.0005)

    threads = [threading.Thread(target=producer, args=(list(range(t, len(jobs), 4)),)) for t in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for j, t in enumerate(tickets):
        assert srv.poll(t, 30000) == gt.GT_OK
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    if policy == gt.GT_SERVE_BATCHED:
        assert st["batches"] >= 2
    if policy == gt.GT_SERVE_SINGLE:
        assert st["batches"] == 0
    assert st["p99_us"] >= st["p50_us"] > 0
    for j, (gi, root) in enumerate(jobs):
        g, og = graphs[gi]
        p_alone, l_alone = g.bfs(root)
        assert np.array_equal(bufs[j][1].cpu().numpy(), l_alone), f"query {j} level differs from gt_bfs alone"
        assert np.array_equal(bufs[j][0].cpu().numpy(), p_alone), f"query {j} parent differs from gt_bfs alone"
        if j % 20 == 0:
            wl, wp = og.bfs(root)
            assert np.array_equal(l_alone, wl) and np.array_equal(p_alone, wp)
    srv.destroy()


def test_budget_admission_and_errors(torch, graphs):
    g, _ = graphs[1]
    small = gt.Server(hbm_budget_bytes=1 << 20)
    with pytest.raises(gt.GtError) as ei:
        small.add_graph(g)
    assert ei.value.code == gt.GT_ENOMEM
    small.destroy()
    srv = gt.Server()
    gid = srv.add_graph(g)
    p = torch.empty(g.n, dtype=torch.int32, device="cuda")
    l = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(gt.GtError) as ei:
        srv.submit(gid, g.n, p, l)  # root out of range
    assert ei.value.code == gt.GT_EINVAL
    with pytest.raises(gt.GtError):
        srv.submit(gid + 5, 0, p, l)  # unknown graph
    hp = np.empty(g.n, dtype=np.int32)
    with pytest.raises(gt.GtError):
        srv.submit(gid, 0, hp, hp)  # host buffers are refused
    with pytest.raises(gt.GtError):
        srv.poll(123456789, 0)  # unknown ticket
    t = srv.submit(gid, 3, p, l)
    rc = srv.poll(t, 0)
    assert rc in (gt.GT_OK, gt.GT_ETIMEOUT)
    if rc == gt.GT_ETIMEOUT:
        assert srv.poll(t, 30000) == gt.GT_OK
    pa, la = g.bfs(3)
    assert np.array_equal(l.cpu().numpy(), la) and np.array_equal(p.cpu().numpy(), pa)
    srv.destroy()


def test_destroy_with_queries_outstanding(torch, graphs):
    g, _ = graphs[0]
    srv = gt.Server(streams=1)
    gid = srv.add_graph(g)
    bufs = [(torch.empty(g.n, dtype=torch.int32, device="cuda"), torch.empty(g.n, dtype=torch.int32, device="cuda"))
            for _ in range(50)]
    for k in range(50):
        srv.submit(gid, k, *bufs[k])
    srv.destroy()  # finishes what is in flight, fails the rest, returns


@pytest.mark.parametrize("scale", [18, 21])
def test_roots_join_a_running_launch(torch, scale):
    # one root starts a batched launch; more roots of the same graph arrive while it runs
    # and join its free lanes at a level boundary; every result equals gt_bfs alone (at
    # scale 21 the core is large enough for the medium-row work list, which then also
    # serves the joined lanes)
    n = 1 << scale
    e = graphgen.rmat_edges(scale, 16, seed=91)
    g = gt.gt_graph_build(e, n)
    cand = graphgen.pick_roots(92, n, 64, g.degree()).tolist()
    joined = 0
    for attempt in range(3):
        srv = gt.Server(streams=1, max_batch_roots=64, policy=gt.GT_SERVE_BATCHED, join_levels=4)
        gid = srv.add_graph(g)
        bufs = [(torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"))
                for _ in cand]
        tickets = [srv.submit(gid, cand[0], *bufs[0])]
        time.sleep(0.0002)
        tickets += [srv.submit(gid, r, *b) for r, b in zip(cand[1:], bufs[1:])]
        for t in tickets:
            assert srv.poll(t, 30000) == gt.GT_OK
        joined = srv.stats()["joined"]
        for r, (p, l) in zip(cand, bufs):
            pa, la = g.bfs(r)
            assert np.array_equal(l.cpu().numpy(), la) and np.array_equal(p.cpu().numpy(), pa), f"root {r}"
        srv.destroy()
        if joined > 0:
            break
    assert joined > 0, "no root joined a running launch in three tries"


def test_lanes_complete_before_their_launch_ends(torch):
    # a long cycle next to a shallow R-MAT component: a batched launch starts from a cycle
    # root (thousands of levels); R-MAT roots arriving meanwhile join its free lanes, end
    # within a few levels, and are written and completed while the launch still runs;
    # every result equals the oracle's
    s, cyc = 13, 6000
    base = 1 << s
    n = base + cyc
    ring = np.arange(cyc, dtype=np.int64) + base
    e = np.concatenate([graphgen.rmat_edges(s, 16, seed=95), np.stack([ring, np.roll(ring, 1)], axis=1)])
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    roots = [base + 17] + graphgen.pick_roots(96, base, 8, og.degree()[:base]).tolist()
    early = joined = 0
    for attempt in range(3):
        srv = gt.Server(streams=1, max_batch_roots=64, policy=gt.GT_SERVE_BATCHED, join_levels=64)
        gid = srv.add_graph(g)
        bufs = [(torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"))
                for _ in roots]
        tickets = [srv.submit(gid, roots[0], *bufs[0])]
        time.sleep(0.0002)
        tickets += [srv.submit(gid, r, *b) for r, b in zip(roots[1:], bufs[1:])]
        for t in tickets:
            assert srv.poll(t, 60000) == gt.GT_OK
        st = srv.stats()
        early, joined = st["early"], st["joined"]
        for r, (p, l) in zip(roots, bufs):
            want_l, want_p = og.bfs(r)
            assert np.array_equal(l.cpu().numpy(), want_l) and np.array_equal(p.cpu().numpy(), want_p), f"root {r}"
        srv.destroy()
        if early > 0:
            break
    assert joined > 0 and early > 0, f"no lane completed before its launch ended in three tries ({joined} joined)"
