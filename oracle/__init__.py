"""FP64 CPU oracle for the Pasur round-by-round CFR solver -- TEST INFRASTRUCTURE ONLY.

This package wraps ``pasur_oracle.c`` (plain C, fp64) through ctypes.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py`` may import it;
the product path (the CUDA library and its binding) never does.  It shares no code with the CUDA
library.  Every function cites the paper passage it restates; what pins each one is listed in
the header of ``pasur_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pasur_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpasur_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: it also builds on the Arm GPU host)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None

P = C.POINTER
i64p = P(C.c_int64)
u64p = P(C.c_uint64)
i32p = P(C.c_int32)
i16p = P(C.c_int16)
i8p = P(C.c_int8)
u8p = P(C.c_uint8)
f64p = P(C.c_double)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.or_splitmix64.argtypes = [C.c_uint64, C.c_int, u64p]
        L.or_xoshiro.argtypes = [C.c_uint64, C.c_int, u64p]
        L.or_xoshiro_state.argtypes = [u64p, C.c_int, u64p]
        L.or_below_seq.argtypes = [C.c_uint64, C.c_int, u64p, u64p]
        L.or_deal.argtypes = [C.c_uint64, u8p]
        L.or_deal.restype = C.c_int
        L.or_subsets_sum.argtypes = [C.c_uint64, C.c_int, u64p, C.c_int64]
        L.or_subsets_sum.restype = C.c_int64
        L.or_legal_actions.argtypes = [C.c_uint64, C.c_uint64, i32p, u64p, C.c_int]
        L.or_legal_actions.restype = C.c_int
        L.or_apply.argtypes = [u64p, i8p, C.c_int, C.c_int, C.c_uint64, C.c_int, u64p, i8p]
        L.or_normalize_score.argtypes = [i16p]
        L.or_round_end.argtypes = [i16p, i8p, i16p]
        L.or_final_leaf.argtypes = [i16p, i8p, C.c_uint64, i16p]
        L.or_final_leaf.restype = C.c_double
        L.or_build_round.argtypes = [u8p, C.c_int, u64p, C.c_int64]
        L.or_build_round.restype = C.c_void_p
        L.or_tree_free.argtypes = [C.c_void_p]
        L.or_tree_sizes.argtypes = [C.c_void_p, i64p, i64p]
        L.or_tree_level.argtypes = [C.c_void_p, C.c_int, i64p, i32p, i32p, u64p, u64p, i8p, i64p]
        L.or_unfold.argtypes = [C.c_void_p, i64p, i16p, i64p]
        L.or_unfold.restype = C.c_int
        L.or_fgt_parents.argtypes = [C.c_void_p, C.c_int, i64p]
        L.or_fgt_parents.restype = C.c_int
        L.or_leaf_utilities_final.argtypes = [C.c_void_p, f64p]
        L.or_leaf_utilities_final.restype = C.c_int
        L.or_next_roots.argtypes = [C.c_void_p, u64p, i64p, i16p, i64p, i64p]
        L.or_next_roots.restype = C.c_int64
        L.or_leaf_utilities_linked.argtypes = [C.c_void_p, i64p, f64p, f64p]
        L.or_leaf_utilities_linked.restype = C.c_int
        L.or_node_values.argtypes = [C.c_void_p, f64p, f64p, C.c_int, f64p]
        L.or_node_values.restype = C.c_int
        L.or_cfr.argtypes = [C.c_void_p, f64p, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double,
                             C.c_double, f64p, f64p, f64p, f64p]
        L.or_cfr.restype = C.c_int
        L.or_cfr_f32.argtypes = [C.c_void_p, f64p, C.c_int, C.c_double, f64p, f64p]
        L.or_cfr_f32.restype = C.c_int
        L.or_root_values.argtypes = [C.c_void_p, f64p, f64p, C.c_int, f64p]
        L.or_root_values.restype = C.c_int
        L.or_count_round.argtypes = [u8p, C.c_int, C.c_uint64, i64p]
        L.or_minimax_rounds.argtypes = [u8p, C.c_int, C.c_uint64, i16p]
        L.or_minimax_rounds.restype = C.c_double
        L.or_philox4x64.argtypes = [u64p, u64p, u64p]
        L.or_selfplay.argtypes = [P(C.c_void_p), C.c_int, P(P(C.c_float)), P(i64p), C.c_int64, C.c_int64,
                                  C.c_uint64, i16p]
        L.or_selfplay.restype = C.c_int
        L.or_outcome_distribution.argtypes = [P(C.c_void_p), C.c_int, P(f64p), P(i64p), C.c_int64, C.c_int,
                                              C.c_int, f64p]
        L.or_outcome_distribution.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t) if a is not None else None


# ---------------------------------------------------------------------------------------------
# Generators and the deal (§Pasur, initial pool rule)
# ---------------------------------------------------------------------------------------------

def splitmix64(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, np.uint64)
    lib().or_splitmix64(seed, n, _p(out, u64p))
    return out


def xoshiro(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, np.uint64)
    lib().or_xoshiro(seed, n, _p(out, u64p))
    return out


def xoshiro_from_state(state4, n: int) -> np.ndarray:
    s = np.asarray(state4, np.uint64).copy()
    out = np.zeros(n, np.uint64)
    lib().or_xoshiro_state(_p(s, u64p), n, _p(out, u64p))
    return out


def below_seq(seed: int, bounds) -> np.ndarray:
    b = np.ascontiguousarray(bounds, np.uint64)
    out = np.zeros(len(b), np.uint64)
    lib().or_below_seq(seed, len(b), _p(b, u64p), _p(out, u64p))
    return out


def deal(seed: int) -> np.ndarray:
    deck = np.zeros(52, np.uint8)
    lib().or_deal(seed, _p(deck, u8p))
    return deck


# ---------------------------------------------------------------------------------------------
# Rules (Table "Capture rules for each card type", Table "Pasur Scoring System")
# ---------------------------------------------------------------------------------------------

def subsets_sum(avail: int, target: int) -> list[int]:
    n = lib().or_subsets_sum(avail, target, None, 0)
    out = np.zeros(max(n, 1), np.uint64)
    lib().or_subsets_sum(avail, target, _p(out, u64p), n)
    return [int(x) for x in out[:n]]


def legal_actions(hand: int, pool: int) -> list[tuple[int, int]]:
    lay = np.zeros(8192, np.int32)
    pick = np.zeros(8192, np.uint64)
    n = lib().or_legal_actions(hand, pool, _p(lay, i32p), _p(pick, u64p), 8192)
    return [(int(lay[i]), int(pick[i])) for i in range(n)]


def apply(state3, rus7, mover: int, lay: int, pick: int, final_round: bool):
    s = np.asarray(state3, np.uint64).copy()
    r = np.asarray(rus7, np.int8).copy()
    so = np.zeros(3, np.uint64)
    ro = np.zeros(7, np.int8)
    lib().or_apply(_p(s, u64p), _p(r, i8p), mover, lay, pick, int(final_round), _p(so, u64p), _p(ro, i8p))
    return so, ro


def normalize_score(score4) -> np.ndarray:
    s = np.asarray(score4, np.int16).copy()
    lib().or_normalize_score(_p(s, i16p))
    return s


def round_end(score4, rus7) -> np.ndarray:
    s = np.asarray(score4, np.int16).copy()
    r = np.asarray(rus7, np.int8).copy()
    o = np.zeros(4, np.int16)
    lib().or_round_end(_p(s, i16p), _p(r, i8p), _p(o, i16p))
    return o


def final_leaf(score4, rus7, pool: int):
    s = np.asarray(score4, np.int16).copy()
    r = np.asarray(rus7, np.int8).copy()
    o = np.zeros(4, np.int16)
    v = lib().or_final_leaf(_p(s, i16p), _p(r, i8p), pool, _p(o, i16p))
    return v, o


def count_round(deck, rnd: int, root_pool: int) -> np.ndarray:
    d = np.asarray(deck, np.uint8).copy()
    out = np.zeros(9, np.int64)
    lib().or_count_round(_p(d, u8p), rnd, root_pool, _p(out, i64p))
    return out


def minimax_rounds(deck, rnd: int, pool: int, score=(0, 0, 0, 0)) -> float:
    """Value-to-go of rounds rnd..5 by direct backward induction (no trees, slots or links)."""
    d = np.asarray(deck, np.uint8).copy()
    s = np.asarray(score, np.int16).copy()
    return lib().or_minimax_rounds(_p(d, u8p), rnd, pool, _p(s, i16p))


# ---------------------------------------------------------------------------------------------
# Round trees, unfolding, between-round links, CFR
# ---------------------------------------------------------------------------------------------

@dataclass
class Level:
    parent: np.ndarray
    nchild: np.ndarray
    lay: np.ndarray
    pick: np.ndarray
    state: np.ndarray   # [n,3] uint64: Alex hand, Bob hand, pool
    rus: np.ndarray     # [n,7] int8
    root_of: np.ndarray


class Tree:
    """An oracle round tree (GT, optionally unfolded into the FGT)."""

    def __init__(self, deck, rnd: int, root_pools):
        self.deck = np.asarray(deck, np.uint8).copy()
        self.round = rnd
        pools = np.asarray(root_pools, np.uint64).copy()
        self._h = lib().or_build_round(_p(self.deck, u8p), rnd, _p(pools, u64p), len(pools))
        if not self._h:
            raise ValueError("or_build_round failed")
        self.unfolded = False

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_tree_free(h)
            self._h = None

    def sizes(self):
        n = np.zeros(9, np.int64)
        q = np.zeros(9, np.int64)
        lib().or_tree_sizes(self._h, _p(n, i64p), _p(q, i64p))
        return n, q

    def level(self, k: int) -> Level:
        n = int(self.sizes()[0][k])
        L = Level(np.zeros(n, np.int64), np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.uint64),
                  np.zeros((n, 3), np.uint64), np.zeros((n, 7), np.int8), np.zeros(n, np.int64))
        lib().or_tree_level(self._h, k, _p(L.parent, i64p), _p(L.nchild, i32p), _p(L.lay, i32p),
                            _p(L.pick, u64p), _p(L.state, u64p), _p(L.rus, i8p), _p(L.root_of, i64p))
        return L

    def unfold(self, score_off, scores) -> np.ndarray:
        so = np.ascontiguousarray(score_off, np.int64)
        sc = np.ascontiguousarray(scores, np.int16).reshape(-1, 4)
        q = np.zeros(9, np.int64)
        if lib().or_unfold(self._h, _p(so, i64p), _p(sc, i16p), _p(q, i64p)) != 0:
            raise ValueError("or_unfold failed")
        self.unfolded = True
        self.score_off, self.scores = so.copy(), sc.copy()
        return q

    def unfold_single(self, score=(0, 0, 0, 0)) -> np.ndarray:
        r = int(self.sizes()[0][0])
        return self.unfold(np.arange(r + 1, dtype=np.int64), np.tile(np.asarray(score, np.int16), (r, 1)))

    def fgt_parents(self, k: int) -> np.ndarray:
        q = self.sizes()[1]
        out = np.zeros(int(q[k]), np.int64)
        if lib().or_fgt_parents(self._h, k, _p(out, i64p)) != 0:
            raise ValueError("or_fgt_parents failed")
        return out

    def leaf_utilities_final(self) -> np.ndarray:
        q = self.sizes()[1]
        out = np.zeros(int(q[8]), np.float64)
        if lib().or_leaf_utilities_final(self._h, _p(out, f64p)) != 0:
            raise ValueError("final-round leaf utilities need an unfolded final-round tree")
        return out

    def next_roots(self):
        npool = C.c_int64(0)
        nroot = lib().or_next_roots(self._h, None, None, None, None, C.byref(npool))
        if nroot < 0:
            raise ValueError("next roots need an unfolded non-final tree")
        pools = np.zeros(npool.value, np.uint64)
        soff = np.zeros(npool.value + 1, np.int64)
        scores = np.zeros((nroot, 4), np.int16)
        lnk = np.zeros(int(self.sizes()[1][8]), np.int64)
        lib().or_next_roots(self._h, _p(pools, u64p), _p(soff, i64p), _p(scores, i16p), _p(lnk, i64p), C.byref(npool))
        return pools, soff, scores, lnk

    def leaf_utilities_linked(self, lnk, u_next) -> np.ndarray:
        q = self.sizes()[1]
        out = np.zeros(int(q[8]), np.float64)
        l = np.ascontiguousarray(lnk, np.int64)
        u = np.ascontiguousarray(u_next, np.float64)
        lib().or_leaf_utilities_linked(self._h, _p(l, i64p), _p(u, f64p), _p(out, f64p))
        return out

    def cfr(self, leaf, iters: int, tau: float = 1e-6, variant: int = 0, alpha=1.5, beta=0.0, gamma=2.0,
            want_rs: bool = False):
        q = self.sizes()[1]
        ne = int(q[1:].sum())
        sb = np.zeros(ne, np.float64)
        U = np.zeros(int(q[0]), np.float64)
        R = np.zeros(ne, np.float64) if want_rs else None
        S = np.zeros(ne, np.float64) if want_rs else None
        lf = np.ascontiguousarray(leaf, np.float64)
        rc = lib().or_cfr(self._h, _p(lf, f64p), iters, tau, variant, alpha, beta, gamma, _p(sb, f64p), _p(U, f64p),
                          _p(R, f64p) if want_rs else None, _p(S, f64p) if want_rs else None)
        if rc != 0:
            raise ValueError("or_cfr failed")
        if want_rs:
            return sb, U, R, S
        return sb, U

    def cfr_f32(self, leaf, iters: int, tau: float = 1e-6):
        """Vanilla CFR in float32 arithmetic (a conditioning probe for the tests, not a reference)."""
        q = self.sizes()[1]
        sb = np.zeros(int(q[1:].sum()), np.float64)
        U = np.zeros(int(q[0]), np.float64)
        lf = np.ascontiguousarray(leaf, np.float64)
        if lib().or_cfr_f32(self._h, _p(lf, f64p), iters, tau, _p(sb, f64p), _p(U, f64p)) != 0:
            raise ValueError("or_cfr_f32 failed")
        return sb, U

    def node_values(self, leaf, mode: int, sigma=None) -> list:
        """Value of every FGT node under `mode` (as root_values), one array per level 0..8."""
        q = self.sizes()[1]
        out = np.zeros(int(q.sum()), np.float64)
        lf = np.ascontiguousarray(leaf, np.float64)
        sg = np.ascontiguousarray(sigma, np.float64) if sigma is not None else None
        if lib().or_node_values(self._h, _p(lf, f64p), _p(sg, f64p), mode, _p(out, f64p)) != 0:
            raise ValueError("or_node_values needs an unfolded tree")
        return np.split(out, np.cumsum(q)[:-1])

    def root_values(self, leaf, mode: int, sigma=None) -> np.ndarray:
        """mode 0 minimax, 1 Alex best response to sigma, 2 Bob best response, 3 both sigma, 4 uniform."""
        q = self.sizes()[1]
        out = np.zeros(int(q[0]), np.float64)
        lf = np.ascontiguousarray(leaf, np.float64)
        sg = np.ascontiguousarray(sigma, np.float64) if sigma is not None else None
        lib().or_root_values(self._h, _p(lf, f64p), _p(sg, f64p), mode, _p(out, f64p))
        return out


MINIMAX, BR_ALEX, BR_BOB, ON_POLICY, UNIFORM = 0, 1, 2, 3, 4


# ---------------------------------------------------------------------------------------------
# Self-play (fair-value simulation; one sampled move per parent, §External Sampling)
# ---------------------------------------------------------------------------------------------


def philox4x64(ctr, key) -> np.ndarray:
    """Philox4x64-10 of one counter block (Salmon et al., SC 2011)."""
    c = np.ascontiguousarray(ctr, np.uint64)
    k = np.ascontiguousarray(key, np.uint64)
    out = np.zeros(4, np.uint64)
    lib().or_philox4x64(_p(c, u64p), _p(k, u64p), _p(out, u64p))
    return out


def _chain(trees, per_round, ctype, np_type):
    arrs = [np.ascontiguousarray(a, np_type) for a in per_round]
    ptrs = (P(ctype) * len(arrs))(*[a.ctypes.data_as(P(ctype)) for a in arrs])
    return arrs, ptrs


def selfplay(trees, sigmas, lnks, root_q: int, n_games: int, seed: int) -> np.ndarray:
    """Final game differences of n_games sampled games from FGT root root_q of trees[0] through
    the rounds of `trees` (the last one final).  sigmas: per round, float32 strategy of every FGT
    edge (levels 1..8); lnks: per non-final round, its leaf-to-next-root links."""
    hs = (C.c_void_p * len(trees))(*[t._h for t in trees])
    sg, sp = _chain(trees, sigmas, C.c_float, np.float32)
    lk, lp = _chain(trees, list(lnks) + [np.zeros(1, np.int64)], C.c_int64, np.int64)
    out = np.zeros(n_games, np.int16)
    if lib().or_selfplay(hs, len(trees), sp, lp, root_q, n_games, seed, _p(out, i16p)) != 0:
        raise ValueError("or_selfplay: invalid arguments")
    return out


def outcome_distribution(trees, sigmas, lnks, root_q: int, lo: int = -128, n_bins: int = 257) -> np.ndarray:
    """Exact probabilities of the final game differences lo .. lo+n_bins-1 when both players
    follow sigmas (float64, laid out as for selfplay)."""
    hs = (C.c_void_p * len(trees))(*[t._h for t in trees])
    sg, sp = _chain(trees, sigmas, C.c_double, np.float64)
    lk, lp = _chain(trees, list(lnks) + [np.zeros(1, np.int64)], C.c_int64, np.int64)
    prob = np.zeros(n_bins, np.float64)
    if lib().or_outcome_distribution(hs, len(trees), sp, lp, root_q, lo, n_bins, _p(prob, f64p)) != 0:
        raise ValueError("or_outcome_distribution: invalid arguments or difference out of range")
    return prob
