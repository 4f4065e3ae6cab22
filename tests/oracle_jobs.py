"""Oracle work for the sampled-root parity tests, run in worker processes.

A sampled check solves a handful of FGT roots of a round with the fp64 oracle (roots are
independent within a round, so a sub-round made of just those roots gives exactly their
values) and compares them with the GPU's values of the same roots.  The oracle part is slow, so
the sample is split into chunks solved by a pool of processes started with "spawn" (safe after
CUDA has been initialised in the parent).  Every oracle input is built here from the deal: the
round's roots come from the oracle's own chain of rounds; the GPU values only come in as the
numbers to compare against.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

import oracle as O

# parity policy (see tests/test_gpu_parity.py)
U_TOL = 1e-5
SIGMA_TOL = 1e-4
MASS_FRAC = 1e-3
NOISE = 1e-6
N_NOISE = 3
COND_TOL = 1e-5
VALUE_TOL = 1e-5
VALUE_CAP = 1e-3


def pool(n: int | None = None):
    n = n or max(1, min(16, os.cpu_count() or 1))
    return mp.get_context("spawn").Pool(n)


def oracle_chain(deck, first: int, last: int, keep=None):
    """The oracle's own chain: for rounds first..last, (pools, score offsets, scores, tree, next)
    with round first from the standalone root and each later round over every root the previous
    one reaches (keep: only that many GT roots of each round below `last`, to bound the cost)."""
    pools = np.array([sum(1 << int(c) for c in deck[:4])], np.uint64)
    soff, sc = np.array([0, 1], np.int64), np.zeros((1, 4), np.int16)
    out = []
    for r in range(first, last + 1):
        if keep is not None and r < last and len(pools) > keep:
            pools, soff, sc = pools[:keep], soff[:keep + 1], sc[:soff[keep]]
        t = O.Tree(deck, r, pools)
        t.unfold(soff, sc)
        nxt = t.next_roots() if r < 5 else None
        out.append(dict(round=r, pools=pools, soff=np.asarray(soff), scores=np.asarray(sc), tree=t, next=nxt))
        if nxt is not None:
            pools, soff, sc = np.asarray(nxt[0], np.uint64), np.asarray(nxt[1]), np.asarray(nxt[2])
    return out


def pick_layout(soff, picks):
    """(roots, slots per root, flat FGT-root indices) of the picked (GT root, slot) pairs in the
    canonical order of a sub-round made of them."""
    by_root: dict = {}
    for g, s in picks:
        by_root.setdefault(int(g), set()).add(int(s))
    roots = sorted(by_root)
    slots = {g: sorted(by_root[g]) for g in roots}
    flat = [int(soff[g] + s) for g in roots for s in slots[g]]
    return roots, slots, np.array(flat, np.int64)


def sub_round(deck, rnd, pools, soff, scores, picks):
    """An oracle tree of round rnd made of the picked (GT root, slot) pairs, in canonical order:
    returns (tree, roots, slots per root, flat FGT-root indices of the picks in that order)."""
    by_root: dict = {}
    for g, s in picks:
        by_root.setdefault(int(g), set()).add(int(s))
    roots = sorted(by_root)
    so, sc, flat = [0], [], []
    for g in roots:
        for s in sorted(by_root[g]):
            sc.append(scores[soff[g] + s])
            flat.append(int(soff[g] + s))
        so.append(len(sc))
    t = O.Tree(deck, rnd, [int(pools[g]) for g in roots])
    t.unfold(np.array(so, np.int64), np.array(sc, np.int16).reshape(-1, 4))
    return t, roots, {g: sorted(by_root[g]) for g in roots}, np.array(flat, np.int64)


def full_edge_index(tree_full, soff, roots, slots):
    """edge_index for an oracle tree of the whole round."""
    return edge_index([tree_full.level(k).root_of for k in range(9)], soff, roots, slots)


def own_mass(ot, S):
    """sum over children of S per FGT edge's parent, laid out per edge (levels 1..8)."""
    q = ot.sizes()[1]
    out = np.zeros_like(S)
    base = 0
    for k in range(1, 9):
        par = ot.fgt_parents(k)
        sums = np.bincount(par, weights=S[base:base + q[k]], minlength=int(q[k - 1]))
        out[base:base + q[k]] = sums[par]
        base += q[k]
    return out


def oracle_sensitivity(ot, leaf_o, sb_o, U_o, T, variant=0, tau=1e-6, keep=None):
    """max |change| of every average strategy and root utility between the fp64 oracle run and
    (a) the same oracle recursion carried out in float32, (b) oracle runs whose leaf values carry
    f32-sized noise (relative and absolute NOISE, seeded signs).  keep (a list, optional)
    receives those runs' average strategies."""
    rng = np.random.default_rng(20250806)
    dp = np.zeros_like(sb_o)
    du = np.zeros_like(U_o)
    if variant == 0:
        sb32, U32 = ot.cfr_f32(leaf_o, T, tau=tau)
        dp = np.abs(sb32 - sb_o)
        du = np.abs(U32 - U_o)
        if keep is not None:
            keep.append(sb32)
    for _ in range(N_NOISE):
        pert = leaf_o * (1 + NOISE * rng.choice([-1.0, 1.0], leaf_o.shape)) + NOISE * rng.choice([-1.0, 1.0], leaf_o.shape)
        sb_p, U_p = ot.cfr(pert, T, tau=tau, variant=variant)
        dp = np.maximum(dp, np.abs(sb_p - sb_o))
        du = np.maximum(du, np.abs(U_p - U_o))
        if keep is not None:
            keep.append(sb_p)
    return dp, du


def check_utilities(U_g, U_o):
    d = np.abs(U_g - U_o)
    assert d.max(initial=0) <= U_TOL, (float(d.max()), int(np.argmax(d)))
    return float(d.max(initial=0))


def check_sigma(ot, leaf_o, sb_g, sb_o, mass, dp, T, label="", perturbed=()):
    """Average strategies: 1e-4 on heavy edges; at an ill-conditioned parent an edge beyond that
    needs value parity instead (see tests/test_gpu_parity.py): the change it makes to the round
    root's value stays within VALUE_TOL plus the largest change the oracle's own perturbed runs
    (perturbed: their average strategies; the float32 recursion and the noisy-leaf runs) make at
    that parent, and never above VALUE_CAP.  Returns (well-conditioned edges, exempted edges,
    their parents, largest strategy difference there, largest value change)."""
    assert np.isfinite(sb_g).all() and (sb_g >= 0).all() and (sb_g <= 1 + 1e-6).all()
    d = np.abs(sb_g - sb_o)
    heavy = mass >= MASS_FRAC * T
    well = heavy & (dp <= COND_TOL)
    ill = heavy & ~well
    assert d[well].max(initial=0) <= SIGMA_TOL, (d[well].max(), int(np.argmax(np.where(well, d, 0))))
    # ill-conditioned edges within the strategy tolerance pass as they are; the others
    # ("exempted") need value parity at their parent
    ill = ill & (d > SIGMA_TOL)
    n_par, dmax, vmax, lmax, rmax = 0, 0.0, 0.0, 0.0, 0.0
    if ill.any():
        q = ot.sizes()[1]
        nv = ot.node_values(leaf_o, O.ON_POLICY, sb_o)
        reach = np.ones(int(q[0]))  # probability of reaching each node when both play sigma-bar
        base = 0
        for k in range(1, 9):
            sl = slice(base, base + int(q[k]))
            par = ot.fgt_parents(k)
            ill_par = np.zeros(int(q[k - 1]), bool)
            ill_par[par[ill[sl]]] = True
            if ill_par.any():
                # the change of the root's value under the oracle's sigma-bar when the GPU's
                # strategy replaces the oracle's at that one parent
                local = np.abs(np.bincount(par, weights=(sb_g[sl] - sb_o[sl]) * nv[k], minlength=int(q[k - 1])))
                dv = reach * local
                ref = np.zeros_like(dv)
                for sp in perturbed:  # what the arithmetic alone does at the same parents
                    ref = np.maximum(ref, reach * np.abs(np.bincount(par, weights=(sp[sl] - sb_o[sl]) * nv[k],
                                                                       minlength=int(q[k - 1]))))
                n_par += int(ill_par.sum())
                lmax = max(lmax, float(local[ill_par].max()))
                vmax = max(vmax, float(dv[ill_par].max()))
                rmax = max(rmax, float(ref[ill_par].max()))
                dmax = max(dmax, float(d[sl][ill[sl]].max()))
                bad = ill_par & ((dv > VALUE_TOL + ref) | (dv > VALUE_CAP))
                assert not bad.any(), (k, float(dv[bad].max()), float(ref[bad].max()))
            reach = reach[par] * sb_o[sl]
            base += int(q[k])
    print(f"[parity{label}] heavy well-conditioned edges {int(well.sum())} (max |d sigma| "
          f"{d[well].max(initial=0):.2e}); ill-conditioned edges beyond the strategy tolerance {int(ill.sum())} at "
          f"{n_par} parents (max |d sigma| {dmax:.2e}, max root-value change {vmax:.2e}, the oracle's own "
          f"perturbed runs up to {rmax:.2e}, max change of the parent's own value {lmax:.2e})")
    return int(well.sum()), int(ill.sum()), n_par, dmax, vmax


def check_sampled(job):
    """Worker: solve the picked FGT roots of one round with the oracle (own leaves: the final
    round's, or the round difference plus the given next-round utilities) and compare with the
    GPU's values of the same roots.  job keys: deck, rnd, pools, soff, scores, picks, T, variant,
    U_g (GPU root utilities of the picks, in sub-round order), sb_g (GPU average strategies of
    the sub-round's edges, in its order), nxt (None, or (pools, score offsets, scores, u) of every
    next-round root with the utilities given to both sides), label.  Returns the statistics of
    check_sigma and the largest root-utility difference."""
    sub, roots, slots, flat = sub_round(job["deck"], job["rnd"], job["pools"], job["soff"], job["scores"], job["picks"])
    if job["nxt"] is None:
        leaf = sub.leaf_utilities_final()
    else:
        npools, nsoff, nsc, u = job["nxt"]
        root_pool = np.repeat(npools, np.diff(nsoff))
        key = {(int(root_pool[i]),) + tuple(int(x) for x in nsc[i]): i for i in range(len(nsc))}
        sp, sso, ssc, sl = sub.next_roots()
        sroot_pool = np.repeat(sp, np.diff(sso))
        u_sub = np.array([u[key[(int(sroot_pool[i]),) + tuple(int(x) for x in ssc[i])]] for i in range(len(ssc))],
                         np.float64)
        leaf = sub.leaf_utilities_linked(sl, u_sub)
    T, variant = job["T"], job["variant"]
    sb_o, U_o, _, S_o = sub.cfr(leaf, T, variant=variant, want_rs=True)
    pert = []
    dp, _ = oracle_sensitivity(sub, leaf, sb_o, U_o, T, variant, keep=pert)
    du = check_utilities(np.asarray(job["U_g"], np.float64), U_o)
    stats = check_sigma(sub, leaf, np.asarray(job["sb_g"], np.float64), sb_o, own_mass(sub, S_o), dp, T,
                        f" {job['label']} max|dU| {du:.2e}", perturbed=pert)
    return dict(label=job["label"], roots=len(roots), fgt_roots=len(flat), edges=int(sub.sizes()[1][1:].sum()),
                du=du, well=stats[0], ill_edges=stats[1], ill_parents=stats[2], ill_dsigma=stats[3], ill_dvalue=stats[4])


def gpu_root_of(gt):
    """Root id of every GT node of a GPU tree, per level (from its exported parents)."""
    n0 = int(gt.pasur_tree_sizes()[0][0])
    out = [np.arange(n0, dtype=np.int64)]
    for k in range(1, 9):
        out.append(out[-1][gt.pasur_export_level(k)["parent"]])
    return out


def edge_index(root_of, soff, roots, slots):
    """Indices, in a round's FGT edge layout (levels 1..8 concatenated; GT-major, slot-minor with
    the root's slots soff[g]..soff[g+1]), of the edges of the sub-round made of the (root, slots)
    pairs, in the sub-round's own order; root_of: root id of every GT node per level."""
    parts, base = [], 0
    for k in range(1, 9):
        ro = root_of[k]
        sl = (soff[ro + 1] - soff[ro]).astype(np.int64)
        off = np.concatenate([[0], np.cumsum(sl)])
        lvl = []
        for g in roots:
            js = np.nonzero(ro == g)[0]
            ss = np.array(slots[g], np.int64)
            lvl.append((off[js][:, None] + ss[None, :]).reshape(-1))
        parts.append(base + np.concatenate(lvl) if lvl else np.zeros(0, np.int64))
        base += int(off[-1])
    return np.concatenate(parts)


def chain_utilities(job):
    """Worker: the oracle's own backward chain over rounds first..5 of a deal (every root of every
    round, each round's leaves from the next round's average utilities, eq. passuputil), T
    iterations per round.  Returns {round: U per FGT root}."""
    deck, first, T = job["deck"], job["first"], job["T"]
    chain = oracle_chain(deck, first, 5)
    out, nxt = {}, None
    for R in reversed(chain):
        t = R["tree"]
        leaf = t.leaf_utilities_final() if R["round"] == 5 else t.leaf_utilities_linked(R["next"][3], nxt)
        _, U = t.cfr(leaf, T)
        out[R["round"]] = U
        nxt = U
    return out
