"""Sharding one deal's backward solve over ranks (paper_2508_06559_gb300/shard.py) on CPU.

Two gloo ranks (127.0.0.1) each solve one contiguous range of every round's GT roots and sum
their round utilities over the ranks (the one exchange per round, eq. passuputil needing the
next round's utilities of every root).  The range solver here is the fp64 oracle on a sub-round
made of the range's roots (roots are independent), so the sharded result must equal the
oracle's unsharded chain exactly.  A rank that fails mid-sweep (an exception raised on the host
between rounds) ends the other rank's next collective with an error instead of a hang.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2508_06559_gb300.shard import partition_roots  # noqa: E402

SEED, FIRST, T = 5, 3, 60


def test_partition_covers_every_root_once():
    rng = np.random.default_rng(1)
    for n, parts in ((0, 3), (1, 4), (7, 2), (50, 8), (200, 3)):
        sizes = rng.integers(1, 1000, n)
        rs = partition_roots(sizes, parts)
        assert len(rs) == parts
        assert rs[0][0] == 0 and sum(c for _, c in rs) == n
        for (f0, c0), (f1, _) in zip(rs, rs[1:]):
            assert f0 + c0 == f1
        if n >= parts:
            tot = [int(sizes[f:f + c].sum()) for f, c in rs]
            assert max(tot) <= sizes.sum() / parts + sizes.max()  # balanced up to one root
    assert partition_roots([0, 0, 0, 0], 2) == [(0, 2), (2, 2)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _oracle_rounds(deck):
    from tests import oracle_jobs as J
    return J.oracle_chain(deck, FIRST, 5)


def _solve_range(deck):
    """The oracle as the range solver: a sub-round made of roots [first, first + count) with all
    their slots; its leaves take the next round's utilities through its own links, mapped to the
    whole next round's roots by (pool, score)."""
    import oracle as O

    def solve(R, u_next, first, count):
        pools, soff, sc = R["pools"], R["soff"], R["scores"]
        u = np.zeros(int(soff[-1]), np.float64)
        if count == 0:
            return u
        a, b = int(soff[first]), int(soff[first + count])
        t = O.Tree(deck, R["round"], pools[first:first + count])
        t.unfold(soff[first:first + count + 1] - a, sc[a:b])
        if R["round"] == 5:
            leaf = t.leaf_utilities_final()
        else:
            npools, nsoff, nsc, _ = R["next"]
            rp = np.repeat(npools, np.diff(nsoff))
            key = {(int(rp[i]),) + tuple(int(x) for x in nsc[i]): i for i in range(len(nsc))}
            sp, sso, ssc, sl = t.next_roots()
            srp = np.repeat(sp, np.diff(sso))
            us = np.array([u_next[key[(int(srp[i]),) + tuple(int(x) for x in ssc[i])]] for i in range(len(ssc))])
            leaf = t.leaf_utilities_linked(sl, us)
        _, U = t.cfr(leaf, T)
        u[a:b] = U
        return u

    return solve


def _rank_main(rank, world, port, out, fail_rank):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import datetime

    import torch
    import torch.distributed as D

    import oracle as O
    from paper_2508_06559_gb300.shard import sharded_backward
    D.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    try:
        deck = O.deal(SEED)
        rounds = _oracle_rounds(deck)
        calls = {"n": 0}

        def sum_over_ranks(u):
            calls["n"] += 1
            if rank == fail_rank and calls["n"] == 2:
                raise RuntimeError("rank failed between rounds")
            t = torch.from_numpy(np.ascontiguousarray(u, np.float64))
            D.all_reduce(t)
            return t.numpy()

        def sizes_of(R):
            t = R["tree"]
            return np.bincount(t.level(8).root_of, minlength=len(R["pools"])) * np.diff(R["soff"])

        try:
            us = sharded_backward(rounds, sizes_of, _solve_range(deck), sum_over_ranks, rank, world, dtype=np.float64)
            out.put((rank, "ok", [u.tolist() for u in us]))
        except Exception as e:  # noqa: BLE001 -- reported to the parent
            out.put((rank, "error", type(e).__name__ + ": " + str(e)[:200]))
    finally:
        try:
            D.destroy_process_group()
        except Exception:  # noqa: BLE001
            pass


def _run(world, fail_rank=-1):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    return res


def test_two_ranks_equal_the_unsharded_oracle_chain():
    from tests import oracle_jobs as J
    import oracle as O
    res = _run(2)
    want = J.chain_utilities(dict(deck=O.deal(SEED), first=FIRST, T=T))
    for rank, status, us in res:
        assert status == "ok", us
        for i, r in enumerate(range(FIRST, 6)):
            assert np.array_equal(np.array(us[i]), want[r]), (rank, r)


def test_failed_rank_ends_the_other_ranks_collective():
    res = _run(2, fail_rank=1)
    assert res[1][1] == "error" and "rank failed" in res[1][2]
    assert res[0][1] == "error"  # the surviving rank's next all-reduce ended with an error
