"""World-size-2 runs on the CPU (gloo backend): the host logic of the N > 1 path.

bench.py runs N independent replicas (weak scaling: every rank scores its own matrix, no
collective on the data path) and reports the whole job's rows/s against the slowest rank's time;
max_over_ranks and job_rows_per_s are run here by two gloo ranks.

The coordinator model of Sec. 3.1.2 (rows sharded across processes, the per-shard sketches summed
once) is checked with the oracle's sketches: each rank sketches its own row range with the rows'
global indices (the hash, sign and Gaussian counters), one all-reduce sums the shard sketches,
and the sum equals the sketch of the whole matrix.  The GPU counterpart of the per-shard sketch is
the streamed entry point's row blocks (tests/test_gpu_streamed.py).
"""
import math
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORLD = 2


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist

    import bench
    from oracle import slso_oracle as O
    from paper_1812_07903_gb300 import inputs

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {"rank": rank}
        out["ms"] = bench.max_over_ranks(1.5 + rank, world, "cpu")
        out["rows_per_s"] = bench.job_rows_per_s(1000, world, out["ms"])

        n, d, s = 3001, 24, 128
        X = inputs.lognormal_rows(n, d, seed=5, dtype=torch.float64).numpy()
        r0, r1 = rank * n // world, (rank + 1) * n // world

        bucket, sign = O.countsketch_hash(n, s, 11)
        part = np.zeros((s, d))
        np.add.at(part, bucket[r0:r1], sign[r0:r1, None] * X[r0:r1])
        t = torch.from_numpy(part)
        dist.all_reduce(t)
        want = O.sketch(X, "countsketch", s, 11)
        out["cs_err"] = float(np.max(np.abs(t.numpy() - want)) / np.max(np.abs(want)))

        G = O.gaussian_block(np.arange(s), np.arange(r0, r1), 13)
        t = torch.from_numpy(G @ X[r0:r1] / math.sqrt(s))
        dist.all_reduce(t)
        want = O.sketch(X, "gaussian", s, 13)
        out["g_err"] = float(np.max(np.abs(t.numpy() - want)) / np.max(np.abs(want)))
        q.put(out)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_sum_shard_sketches():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in range(WORLD)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in results:
        assert r["ms"] == 2.5  # the slowest rank's time, on every rank
        assert r["rows_per_s"] == WORLD * 1000 / 2.5e-3
        assert r["cs_err"] < 1e-14
        assert r["g_err"] < 1e-13
