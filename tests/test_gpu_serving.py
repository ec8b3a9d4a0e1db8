"""Serving (continuous batching): each job's result is the same alone and in the mix.

A mixed batch of leverage jobs (CountSketch, SRHT, Gaussian; uneven n and d; float32 and
bfloat16 paths) and sketched-SVD jobs is first run job by job through the direct entry points,
then submitted at once to a server whose memory budget forces queueing.  Every output must be
bitwise identical: the kernels are deterministic, and concurrent jobs share no state.
"""
import numpy as np
import pytest
import torch

from paper_1812_07903_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _jobs():
    rng = np.random.default_rng(5)
    out = []
    for j in range(14):
        n = int(round(2 ** rng.uniform(11, 15)))
        d = int(rng.choice([16, 64, 100, 128]))
        kind = ["countsketch", "srht", "gaussian"][j % 3]
        s = inputs.serving_sketch_rows(n, d, kind)
        compute = "bf16" if j % 4 == 3 else "f32"
        X = inputs.gaussian_mixture(n, d, seed=10000 + j, device="cuda")
        out.append(dict(X=X, kind=kind, s=s, k=64 if j % 5 else 0, seed_S=20000 + j, seed_Pi=30000 + j,
                        compute=compute))
    return out


def test_results_alone_equal_results_in_the_mix():
    jobs = _jobs()
    svd_inputs = [torch.randn(600 + 100 * i, 40 + 13 * i, dtype=torch.float64, device="cuda") for i in range(3)]
    alone = []
    for jb in jobs:
        sc, info = api.leverage(jb["X"], jb["kind"], jb["s"], jb["k"], jb["seed_S"], jb["seed_Pi"],
                                compute=jb["compute"])
        alone.append((sc.clone(), api.order(sc).clone(), info["rank"]))
    alone_svd = [api.sketched_svd(SX)[:3] for SX in svd_inputs]
    torch.cuda.synchronize()

    srv = api.Server(slots=4, mem_budget_bytes=96 << 20)
    tickets = [srv.submit_leverage(jb["X"], jb["kind"], jb["s"], jb["k"], jb["seed_S"], jb["seed_Pi"],
                                   compute=jb["compute"]) for jb in jobs]
    svd_tickets = [srv.submit_sketched_svd(SX) for SX in svd_inputs]
    lat = []
    for t, (sc0, o0, r0) in zip(tickets, alone):
        st, info, times, (sc, o) = srv.poll(t)
        assert st == 0 and info["rank"] == r0
        assert torch.equal(sc, sc0) and torch.equal(o, o0)
        lat.append(times[2])
    for t, (sg0, V0, R0) in zip(svd_tickets, alone_svd):
        st, info, times, (sg, V, R) = srv.poll(t)
        assert st == 0
        assert torch.equal(sg, sg0) and torch.equal(V, V0) and torch.equal(R, R0)
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(jobs) + len(svd_inputs) and stats["queued"] == 0
    assert all(x > 0 for x in lat)


def test_admission_refuses_a_job_larger_than_the_budget():
    srv = api.Server(slots=2, mem_budget_bytes=1 << 20)
    X = inputs.gaussian_mixture(50000, 128, seed=1, device="cuda")
    with pytest.raises(RuntimeError, match="BUSY"):
        srv.submit_leverage(X, "countsketch", 4096, 64, 1, 2)
    srv.close()


def test_invalid_job_is_rejected_at_submit():
    srv = api.Server(slots=1, mem_budget_bytes=1 << 30)
    X = inputs.gaussian_mixture(1000, 64, seed=1, device="cuda")
    with pytest.raises(RuntimeError, match="SHAPE"):
        srv.submit_leverage(X, "countsketch", 32, 16, 1, 2)  # s < d
    srv.close()


def test_repeated_shapes_replay_captured_graphs():
    """A shape's first job runs direct, its second is captured into a graph, later ones replay
    that graph with their own X, scores and order (updated in place); results equal the direct
    entry points bit for bit.  The shapes' JL widths (k rounded up to 32) differ, so queued jobs
    never share a grouped score launch here, whatever the timing."""
    shapes = [(20000, 64, "countsketch", 1024, 32), (9000, 100, "srht", 512, 0), (12000, 48, "gaussian", 256, 40)]
    srv = api.Server(slots=1, mem_budget_bytes=1 << 30)
    want, tickets = [], []
    for rep in range(3):
        for i, (n, d, kind, s, k) in enumerate(shapes):
            X = inputs.gaussian_mixture(n, d, seed=100 * rep + i, device="cuda")
            sc, _ = api.leverage(X, kind, s, k, 7, 8)
            want.append((sc.clone(), api.order(sc).clone()))
            tickets.append(srv.submit_leverage(X, kind, s, k, 7, 8))
    for t, (sc0, o0) in zip(tickets, want):
        st, info, times, (sc, o) = srv.poll(t)
        assert st == 0 and torch.equal(sc, sc0) and torch.equal(o, o0)
    c = srv.counters()
    srv.close()
    assert c["direct"] == len(shapes) and c["graphs_new"] == len(shapes) and c["graphs_updated"] == len(shapes)


def test_queued_small_jobs_share_a_grouped_launch():
    """Small float32 jobs queued behind a long one are admitted together and scored by one grouped
    tensor-core launch (the counters show it); every result equals its direct call bit for bit."""
    blocker = inputs.gaussian_mixture(1 << 20, 256, seed=1, device="cuda")
    small = []
    for j in range(6):
        n = [5000, 20000, 777, 65536, 12345, 3000][j]
        d = [64, 100, 36, 128, 64, 96][j]
        kind = ["countsketch", "srht", "gaussian"][j % 3]
        X = inputs.gaussian_mixture(n, d, seed=200 + j, device="cuda")
        small.append(dict(X=X, kind=kind, s=inputs.serving_sketch_rows(n, d, kind), seed_S=40 + j, seed_Pi=50 + j))
    want = []
    for jb in small:
        sc, info = api.leverage(jb["X"], jb["kind"], jb["s"], 64, jb["seed_S"], jb["seed_Pi"], compute="f32")
        want.append((sc.clone(), api.order(sc).clone(), info["rank"]))
    torch.cuda.synchronize()
    srv = api.Server(slots=1, mem_budget_bytes=4 << 30)
    tb = srv.submit_leverage(blocker, "countsketch", 8192, 64, 3, 4)
    tickets = [srv.submit_leverage(jb["X"], jb["kind"], jb["s"], 64, jb["seed_S"], jb["seed_Pi"]) for jb in small]
    assert srv.poll(tb)[0] == 0
    for t, (sc0, o0, r0) in zip(tickets, want):
        st, info, times, (sc, o) = srv.poll(t)
        assert st == 0 and info["rank"] == r0
        assert torch.equal(sc, sc0) and torch.equal(o, o0)
    c = srv.counters()
    srv.close()
    assert c["group_launches"] >= 1 and c["grouped_jobs"] >= 2
