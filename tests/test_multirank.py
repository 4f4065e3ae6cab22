"""The benchmark's multi-process path on CPU: two ranks over gloo (127.0.0.1), as under
torchrun.  Ranks are independent replicas: each solves its own deals (no two ranks share a
deal), the timing takes the maximum over ranks, and the whole-job rate is the sum of every rank's
node-updates over the slowest rank's time.  The reference arm does no work on ranks other than 0.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as D
    import bench
    D.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = {w: bench.rank_deal_seeds(w, 7, rank) for w in bench.WORKLOADS}
        gathered = [None] * world
        D.all_gather_object(gathered, seeds)
        mx = bench.reduce_over_ranks(D, 10.0 * (rank + 1), "max", "cpu")
        sm = bench.reduce_over_ranks(D, 10.0 * (rank + 1), "sum", "cpu")
        ref = bench.run_reference(type("A", (), {"workload": "final_round", "seed": 0, "iters": 10, "steps": 1,
                                                 "warmup": 0})(), rank, world) if rank else "skipped"
        D.barrier()
        out.put((rank, gathered, mx, sm, ref))
    finally:
        D.destroy_process_group()


def test_two_ranks_replicas_and_reductions():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (_, gathered, mx0, sm0, _), (_, _, mx1, sm1, ref1) = res
    assert mx0 == mx1 == 20.0 and sm0 == sm1 == 30.0
    for w in gathered[0]:
        a, b = set(gathered[0][w]), set(gathered[1][w])
        assert a and b and not (a & b), w          # every rank its own deals
        assert len(a) == len(b)                    # same work shape per rank (weak scaling)
    assert gathered[0]["full_game"] == [7] and gathered[1]["full_game"] == [8]
    assert ref1 is None                            # the reference arm runs on rank 0 only


def test_job_rate_sums_ranks_over_the_slowest():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(3e10 + 5e10, 0.25) == pytest.approx(3.2e11)
    assert bench.reduce_over_ranks(None, 4.0, "max", "cpu") == 4.0


def test_size_histogram_counts_per_decade():
    sys.path.insert(0, ROOT)
    import bench
    h = bench.size_histogram([110_651, 999_999, 1_000_000, 6_474_184, 2_000_000])
    assert h["deals"] == 5 and h["min"] == 110_651 and h["max"] == 6_474_184
    assert h["median"] == 1_000_000
    assert h["per_decade"] == {"1e5-1e6": 2, "1e6-1e7": 3}
