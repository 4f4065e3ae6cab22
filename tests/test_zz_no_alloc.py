"""The allocation-free offsets entry point (pasur_move_offsets_noalloc) against the allocating path.

pasur_build_round turns every node's number of legal moves into CSR child offsets with a scan
whose scratch it allocates; pasur_move_offsets_noalloc does the same step for callers that cannot
allocate device memory (an application that gives all GPU memory to its own arena, a plug-in
inside a host program that owns the allocator, code that must not risk an out-of-memory failure
mid-run), with its scratch in a fixed array inside the library.  Here both see the same counts:
the move counts of every level of real round trees, exported from pasur_build_round.  The
offsets of the allocation-free call, expanded into parent indices, must equal the parents that
pasur_build_round emitted with its own offsets, bit for bit, on two calls in a row (the second
call reuses the array the first one left behind).  This file is collected last so that a failure
here cannot hide any other test.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_06559_gb300 import build as B
    from paper_2508_06559_gb300 import pasur as P
    B.build()
    c = P.Ctx(0)
    yield c
    c.close()


def test_noalloc_offsets_match_build_round(ctx):
    import torch

    from paper_2508_06559_gb300 import pasur as P
    deck = O.deal(0)
    t4 = O.Tree(deck, 4, [mask_ids(deck[:4])])
    t4.unfold_single()
    pools, _, _, _ = t4.next_roots()
    tree = ctx.pasur_build_round(deck, 5, pools)  # 37 roots, levels of 37 .. 30,577 nodes
    sizes = tree.pasur_tree_sizes()[0]
    for k in range(8):
        counts = tree.pasur_export_level(k)["nchild"]
        parents = tree.pasur_export_level(k + 1)["parent"]
        cd = torch.from_numpy(counts.astype(np.int32)).cuda()
        for call in range(2):
            off = torch.full((len(counts) + 1,), -7, dtype=torch.int64, device="cuda")
            P.pasur_move_offsets_noalloc(cd, off)
            torch.cuda.synchronize()
            o = off.cpu().numpy()
            assert o[0] == 0 and o[-1] == sizes[k + 1], (k, call)
            expanded = np.repeat(np.arange(len(counts)), np.diff(o))
            assert (expanded == parents).all(), (k, call)


def test_noalloc_offsets_large_and_limits(ctx):
    import torch

    from paper_2508_06559_gb300 import pasur as P
    n = 4_194_303  # the documented maximum: every tile of the fixed scratch array in use
    rng = np.random.default_rng(3)
    counts = rng.integers(0, 9, n).astype(np.int32)
    cd = torch.from_numpy(counts).cuda()
    expect = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
    for _ in range(2):
        off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        P.pasur_move_offsets_noalloc(cd, off)
        torch.cuda.synchronize()
        assert (off.cpu().numpy() == expect).all()
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    off1 = torch.full((1,), 5, dtype=torch.int64, device="cuda")
    P.pasur_move_offsets_noalloc(empty, off1)
    torch.cuda.synchronize()
    assert int(off1.item()) == 0
    too_big = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    off2 = torch.empty(n + 2, dtype=torch.int64, device="cuda")
    with pytest.raises(P.PasurError) as e:
        P.pasur_move_offsets_noalloc(too_big, off2)
    assert e.value.code == P.PASUR_EOVERFLOW


def test_noalloc_rejects_wrong_buffers(ctx):
    """Wrong tensors are refused before any kernel runs: a host buffer, the wrong element type, an
    offsets buffer shorter than n+1 (the C call has no capacity argument), a strided view."""
    import torch

    from paper_2508_06559_gb300 import pasur as P
    n = 1000
    good_c = torch.ones(n, dtype=torch.int32, device="cuda")
    good_o = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    cases = [
        (good_c.cpu(), good_o),                                            # host counts
        (good_c, good_o.cpu()),                                            # host offsets
        (good_c.to(torch.int64), good_o),                                  # int64 counts
        (good_c, good_o.to(torch.int32)),                                  # int32 offsets
        (good_c, good_o[:n]),                                              # offsets too short
        (torch.ones(2 * n, dtype=torch.int32, device="cuda")[::2], good_o),  # strided counts
    ]
    for c, o in cases:
        with pytest.raises(P.PasurError) as e:
            P.pasur_move_offsets_noalloc(c, o)
        assert e.value.code == P.PASUR_EINVAL
    # a host pointer given straight to the C entry point is refused too
    import ctypes

    h = np.zeros(n + 1, np.int64)
    rc = P.load().pasur_move_offsets_noalloc(ctypes.c_void_p(good_c.data_ptr()), n, ctypes.c_void_p(h.ctypes.data),
                                            None)
    assert rc == P.PASUR_EINVAL
    # the good pair still works after the refusals, on torch's current (non-default) stream
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        P.pasur_move_offsets_noalloc(good_c, good_o)
    s.synchronize()
    assert (good_o.cpu().numpy() == np.arange(n + 1)).all()
