"""Host-side logic of the multi-GPU benchmark (independent replicas), run as
two gloo ranks on the CPU: each rank mines its own batch, timings are
reduced to the slowest rank, and the whole-job rate counts every rank's
pairs."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_1509_08639_gb300 import synth
    dist.init_process_group("gloo")
    try:
        ws_, rank_, _ = bench.dist_env()
        seed = bench.rank_seed(2, rank_)
        w = synth.workload(2, n_pairs=40, seed=seed)
        local_ms = 10.0 + 5.0 * rank_            # rank 1 is slower
        slowest = bench.max_over_ranks(local_ms, ws_)
        rate = bench.whole_job_rate(w.batch.n_pairs, ws_, slowest / 1e3)
        q.put((rank_, seed, int(w.batch.tokens.sum()), slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(ws)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    out.sort()
    (r0, s0, tok0, m0, v0), (r1, s1, tok1, m1, v1) = out
    assert s0 is None and s1 is not None           # distinct, deterministic batches
    assert tok0 != tok1
    assert m0 == m1 == 15.0                        # max over ranks
    assert v0 == v1 == pytest.approx(2 * 40 / 0.015)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.rank_seed(2, 0) is None and bench.rank_seed(2, 3) == 1508 + 2 + 3000
